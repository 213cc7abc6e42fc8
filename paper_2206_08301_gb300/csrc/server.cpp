// Serving loop for CP-ALS requests: continuous batching under an HBM budget.
//
// The server owns one device arena (the budget, one cudaMalloc at creation)
// and a set of slots, each with its own CUDA stream.  A submitted request
// waits in a FIFO until a slot is free and the arena can place its footprint
// (X, factors, generating factors, lambda, fits, the CP-ALS workspace); it is
// then admitted: on its slot's stream its X is generated from its seed on the
// device, its CP-ALS sweeps are enqueued, and an event marks the end.
// Requests that arrive while others run are admitted as soon as a slot and
// memory free up, so the work of several requests overlaps on the device.
// poll() retires finished requests (fit and lambda read back, memory and slot
// released) and admits waiting ones.  Nothing here blocks on the device except
// the small result copies of a request that has already finished.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// First-fit allocator over [0, size) with coalescing of freed neighbours.
class Arena {
  public:
    explicit Arena(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t noff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[noff] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t largest() const {
        size_t m = 0;
        for (auto &kv : free_) m = kv.second > m ? kv.second : m;
        return m;
    }

  private:
    std::map<size_t, size_t> free_;
};

struct Request {
    int64_t id = 0;
    int order = 0;
    int64_t dims[DEINSUM_MAX_ORDER] = {0};
    int rank = 0, sweeps = 0, cp_rank = 0;
    uint64_t seed = 0;
    double noise = 0.0;
    std::vector<float> cpf;    // generating factors, concatenated by mode
    std::vector<float> init;   // initial factors, concatenated by mode
    bool want_factors = false;
    double arrival = 0.0, admit = 0.0, done = 0.0;
    int status = 0;
    double gen_ms = 0.0;
    std::vector<double> fits, lambda;
    std::vector<float> factors;
    bool finished = false;
    // device placement
    size_t off = 0, bytes = 0;
    deinsum_cpals_t cp = nullptr;
    int slot = -1;
    float *dX = nullptr;
    float *dF[DEINSUM_MAX_ORDER] = {nullptr};
    float *dA[DEINSUM_MAX_ORDER] = {nullptr};
    double *dLam = nullptr, *dFits = nullptr;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr, g0 = nullptr, g1 = nullptr;
    double *host = nullptr;  // pinned: fits (<= 4096) then lambda (<= 64)
    Request *req = nullptr;
};

constexpr int kMaxSweeps = 4096;

}  // namespace

struct deinsum_server_s {
    char *arena_ptr = nullptr;
    size_t arena_bytes = 0;
    std::unique_ptr<Arena> arena;
    deinsum_prec prec = DEINSUM_PREC_SPLIT_BF16;
    std::vector<Slot> slots;
    std::deque<Request *> waiting;
    std::unordered_map<int64_t, std::unique_ptr<Request>> all;
    int64_t next_id = 1;
};

namespace {

// Device footprint of a request (each part 1024-byte aligned) -- needs the
// CP-ALS handle for the size of its workspace.
size_t footprint(const Request &r, size_t cp_ws) {
    int64_t nx = 1;
    size_t b = 0;
    for (int m = 0; m < r.order; ++m) {
        nx *= r.dims[m];
        b += up(size_t(r.dims[m]) * r.rank * 4, 1024) + up(size_t(r.dims[m]) * r.cp_rank * 4, 1024);
    }
    b += up(size_t(nx) * 4, 1024) + up(size_t(r.rank) * 8, 1024) + up(size_t(r.sweeps) * 8, 1024);
    return b + up(cp_ws, 1024);
}

// Place and start a request on slot `si` (its stream).  Returns false if the
// arena cannot place it now (it stays queued); sets r.status on hard errors.
bool admit(deinsum_server_s *s, Request *r, int si) {
    Slot &sl = s->slots[size_t(si)];
    if (!r->cp) {
        deinsum_status st = deinsum_cpals_create(r->order, r->dims, r->rank, s->prec, &r->cp);
        if (st != DEINSUM_OK) {
            r->status = st;
            return true;
        }
    }
    size_t cpws = 0;
    deinsum_status st = deinsum_cpals_workspace_bytes(r->cp, &cpws);
    if (st != DEINSUM_OK) {
        r->status = st;
        return true;
    }
    const size_t need = footprint(*r, cpws);
    if (need > s->arena_bytes) {
        r->status = DEINSUM_ERR_OOM;
        return true;
    }
    size_t off = 0;
    if (!s->arena->alloc(need, &off)) return false;
    r->off = off;
    r->bytes = need;
    r->slot = si;
    r->admit = now_s();
    char *p = s->arena_ptr + off;
    auto take = [&](size_t n) {
        char *q = p;
        p += up(n, 1024);
        return q;
    };
    int64_t nx = 1;
    for (int m = 0; m < r->order; ++m) nx *= r->dims[m];
    r->dX = reinterpret_cast<float *>(take(size_t(nx) * 4));
    for (int m = 0; m < r->order; ++m) {
        r->dF[m] = reinterpret_cast<float *>(take(size_t(r->dims[m]) * r->rank * 4));
        r->dA[m] = reinterpret_cast<float *>(take(size_t(r->dims[m]) * r->cp_rank * 4));
    }
    r->dLam = reinterpret_cast<double *>(take(size_t(r->rank) * 8));
    r->dFits = reinterpret_cast<double *>(take(size_t(r->sweeps) * 8));
    char *ws = take(cpws);
    cudaStream_t str = sl.stream;
    size_t fo = 0, ao = 0;
    for (int m = 0; m < r->order; ++m) {
        const size_t nf = size_t(r->dims[m]) * r->rank, na = size_t(r->dims[m]) * r->cp_rank;
        cudaMemcpyAsync(r->dA[m], r->cpf.data() + ao, na * 4, cudaMemcpyHostToDevice, str);
        cudaMemcpyAsync(r->dF[m], r->init.data() + fo, nf * 4, cudaMemcpyHostToDevice, str);
        fo += nf;
        ao += na;
    }
    cudaEventRecord(sl.g0, str);
    st = deinsum_gen_cp_f32(r->seed, r->order, r->dims, r->cp_rank, r->dA, r->noise, r->dX, str);
    cudaEventRecord(sl.g1, str);
    if (st == DEINSUM_OK) st = deinsum_cpals_bind_workspace(r->cp, ws, cpws, str);
    if (st == DEINSUM_OK) st = deinsum_cpals_run(r->cp, r->dX, r->dF, r->dLam, r->sweeps, r->dFits, str);
    if (st == DEINSUM_OK) {
        cudaMemcpyAsync(sl.host, r->dFits, size_t(r->sweeps) * 8, cudaMemcpyDeviceToHost, str);
        cudaMemcpyAsync(sl.host + kMaxSweeps, r->dLam, size_t(r->rank) * 8, cudaMemcpyDeviceToHost, str);
    }
    cudaEventRecord(sl.done, str);
    r->status = st;
    sl.req = r;
    return true;
}

void retire(deinsum_server_s *s, Slot &sl) {
    Request *r = sl.req;
    r->done = now_s();
    if (r->status == DEINSUM_OK) {
        r->fits.assign(sl.host, sl.host + r->sweeps);
        r->lambda.assign(sl.host + kMaxSweeps, sl.host + kMaxSweeps + r->rank);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, sl.g0, sl.g1) == cudaSuccess) r->gen_ms = ms;
        deinsum_status st = deinsum_cpals_status(r->cp);
        if (st != DEINSUM_OK) r->status = st;
        if (r->want_factors) {
            size_t total = 0;
            for (int m = 0; m < r->order; ++m) total += size_t(r->dims[m]) * r->rank;
            r->factors.resize(total);
            size_t fo = 0;
            for (int m = 0; m < r->order; ++m) {
                const size_t nf = size_t(r->dims[m]) * r->rank;
                cudaMemcpy(r->factors.data() + fo, r->dF[m], nf * 4, cudaMemcpyDeviceToHost);
                fo += nf;
            }
        }
    }
    deinsum_cpals_destroy(r->cp);
    r->cp = nullptr;
    s->arena->release(r->off, r->bytes);
    r->finished = true;
    r->slot = -1;
    sl.req = nullptr;
}

}  // namespace

extern "C" {

double deinsum_server_clock(void) { return now_s(); }

deinsum_status deinsum_server_create(size_t hbm_budget_bytes, int slots, deinsum_prec prec, deinsum_server_t *out) {
    if (!out || slots < 1 || slots > 64 || hbm_budget_bytes < (size_t(1) << 20)) return DEINSUM_ERR_INVALID;
    *out = nullptr;
    deinsum_server_s *s = new (std::nothrow) deinsum_server_s();
    if (!s) return DEINSUM_ERR_OOM;
    s->prec = prec;
    void *p = nullptr;
    cudaError_t e = deinsum::counted_malloc(&p, hbm_budget_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return e == cudaErrorMemoryAllocation ? DEINSUM_ERR_OOM : DEINSUM_ERR_CUDA;
    }
    s->arena_ptr = static_cast<char *>(p);
    s->arena_bytes = hbm_budget_bytes;
    s->arena.reset(new Arena(hbm_budget_bytes));
    s->slots.resize(size_t(slots));
    for (auto &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreate(&sl.g0) != cudaSuccess || cudaEventCreate(&sl.g1) != cudaSuccess ||
            deinsum::counted_malloc_host(reinterpret_cast<void **>(&sl.host), (kMaxSweeps + 64) * sizeof(double)) != cudaSuccess) {
            deinsum_server_destroy(s);
            return DEINSUM_ERR_CUDA;
        }
    }
    *out = s;
    return DEINSUM_OK;
}

deinsum_status deinsum_server_submit(deinsum_server_t s, const deinsum_request_t *q, int64_t *id) {
    if (!s || !q || !id || !q->cp_factors || !q->init_factors) return DEINSUM_ERR_INVALID;
    if (q->order < 2 || q->order > DEINSUM_MAX_ORDER || q->rank < 1 || q->rank > 64 || q->cp_rank < 1 ||
        q->sweeps < 1 || q->sweeps > kMaxSweeps)
        return DEINSUM_ERR_SHAPE;
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return DEINSUM_ERR_OOM;
    r->id = s->next_id++;
    r->order = q->order;
    r->rank = q->rank;
    r->sweeps = q->sweeps;
    r->cp_rank = q->cp_rank;
    r->seed = q->seed;
    r->noise = q->noise;
    r->arrival = q->arrival_s;
    r->want_factors = q->want_factors != 0;
    for (int m = 0; m < q->order; ++m) {
        if (q->dims[m] < 1 || !q->cp_factors[m] || !q->init_factors[m]) return DEINSUM_ERR_INVALID;
        r->dims[m] = q->dims[m];
        r->cpf.insert(r->cpf.end(), q->cp_factors[m], q->cp_factors[m] + q->dims[m] * q->cp_rank);
        r->init.insert(r->init.end(), q->init_factors[m], q->init_factors[m] + q->dims[m] * q->rank);
    }
    *id = r->id;
    s->waiting.push_back(r.get());
    s->all.emplace(r->id, std::move(r));
    return DEINSUM_OK;
}

deinsum_status deinsum_server_poll(deinsum_server_t s, int *n_active, int *n_waiting) {
    if (!s) return DEINSUM_ERR_INVALID;
    for (auto &sl : s->slots) {
        if (!sl.req) continue;
        const cudaError_t e = cudaEventQuery(sl.done);
        if (e == cudaSuccess) {
            retire(s, sl);
        } else if (e != cudaErrorNotReady) {
            cudaGetLastError();
            sl.req->status = DEINSUM_ERR_CUDA;
            retire(s, sl);
        }
    }
    // FIFO admission: the head waits until a slot and enough arena are free
    while (!s->waiting.empty()) {
        int free_slot = -1;
        for (size_t i = 0; i < s->slots.size(); ++i)
            if (!s->slots[i].req) {
                free_slot = int(i);
                break;
            }
        if (free_slot < 0) break;
        Request *r = s->waiting.front();
        if (!admit(s, r, free_slot)) break;
        s->waiting.pop_front();
        if (r->status != DEINSUM_OK && s->slots[size_t(free_slot)].req != r) {
            // refused before launch (too large, bad plan): finished with its status
            r->admit = r->done = now_s();
            if (r->cp) {
                deinsum_cpals_destroy(r->cp);
                r->cp = nullptr;
            }
            r->finished = true;
        }
    }
    int act = 0;
    for (auto &sl : s->slots) act += sl.req ? 1 : 0;
    if (n_active) *n_active = act;
    if (n_waiting) *n_waiting = int(s->waiting.size());
    return DEINSUM_OK;
}

deinsum_status deinsum_server_take(deinsum_server_t s, int64_t id, deinsum_result_t *res, double *fits,
                                   double *lambda, float *factors) {
    if (!s || !res) return DEINSUM_ERR_INVALID;
    auto it = s->all.find(id);
    if (it == s->all.end() || !it->second->finished) return DEINSUM_ERR_INVALID;
    Request &r = *it->second;
    res->id = r.id;
    res->status = r.status;
    res->arrival_s = r.arrival;
    res->admit_s = r.admit;
    res->done_s = r.done;
    res->gen_ms = r.gen_ms;
    res->sweeps = r.sweeps;
    res->fit = r.fits.empty() ? 0.0 : r.fits.back();
    if (fits && !r.fits.empty()) std::memcpy(fits, r.fits.data(), r.fits.size() * sizeof(double));
    if (lambda && !r.lambda.empty()) std::memcpy(lambda, r.lambda.data(), r.lambda.size() * sizeof(double));
    if (factors && !r.factors.empty()) std::memcpy(factors, r.factors.data(), r.factors.size() * sizeof(float));
    s->all.erase(it);
    return DEINSUM_OK;
}

void deinsum_server_destroy(deinsum_server_t s) {
    if (!s) return;
    for (auto &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.req && sl.req->cp) deinsum_cpals_destroy(sl.req->cp);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.g0) cudaEventDestroy(sl.g0);
        if (sl.g1) cudaEventDestroy(sl.g1);
        if (sl.host) cudaFreeHost(sl.host);
    }
    for (auto &kv : s->all)
        if (kv.second->cp) deinsum_cpals_destroy(kv.second->cp);
    if (s->arena_ptr) cudaFree(s->arena_ptr);
    delete s;
}

}  // extern "C"
