"""Host-side checks of the C ABI (no compute calls, no GPU needed).

The library must load, export every function include/deinsum.h declares, and
plan (parse + classify, host only) the paper's Table IV patterns while
rejecting everything else with the documented status codes.
"""
import ctypes
import os
import re

import pytest

import paper_2206_08301_gb300 as dz
from paper_2206_08301_gb300 import build as dbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "deinsum.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(dz.library_path()):
        dbuild.build()
    return dz.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(deinsum_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("deinsum_plan", "deinsum_execute", "deinsum_workspace_size", "deinsum_last_device_status",
                 "deinsum_destroy", "deinsum_status_string", "deinsum_plan_info"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(dz.library_path())
    for name in declared_functions():
        assert hasattr(raw, name), f"{name} declared but not exported"


@pytest.mark.parametrize("spec,kind,mode", [
    ("ijk,ja,ka->ia", "mttkrp", 0),     # Table IV MTTKRP-O3-M0
    ("ijk,ia,ka->ja", "mttkrp", 1),     # MTTKRP-O3-M1
    ("ijk,ia,ja->ka", "mttkrp", 2),     # MTTKRP-O3-M2
    ("ijklm,ja,ka,la,ma->ia", "mttkrp", 0),
    ("ijklm,ia,ja,la,ma->ka", "mttkrp", 2),
    ("ijklm,ia,ja,ka,la->ma", "mttkrp", 4),
    ("ijklm,jb,kc,ld,me->ibcde", "ttmc", 0),   # TTMc-O5-M0
    ("ijkl,jb,kc,ld->ibcd", "ttmc", 0),
    ("ijk,ib,jc->bck", "ttmc", 2),
])
def test_plan_classifies_table_iv_patterns(lib, spec, kind, mode):
    letters = []
    for c in spec:
        if c.isalpha() and c not in letters:
            letters.append(c)
    p = dz.Plan(spec, [5] * len(letters))
    assert p.kind == kind and p.mode == mode
    assert p.workspace_size() == 0  # nothing allocated before the first execute


@pytest.mark.parametrize("spec,status", [
    ("ijk,ja,ka", 1),             # no output
    ("ijk,ja,ka->i a", 2),        # spaces are removed -> "ia"... handled below
    ("ij1,ja->ia", 1),            # bad character
    ("ijk,ja,ka,al->ia", 2),      # MTTKRP + MM with the rank letter kept in the output
    ("ijk,ja,ka,al,lm->im", 2),   # MTTKRP + two matrix products: not offered
    ("ij,jk,kl->il", 2),          # 2MM chain: not offered
    ("iik,ia,ka->ia", 2),         # diagonal of X
    ("ijk,ja,kb->iba", 2),        # TTMc with permuted output modes: not offered
    ("ijk,ja,ka->ai", 2),         # transposed MTTKRP output
    ("ijk,ja,ka->iz", 2),         # output letter missing from the inputs
])
def test_plan_rejects(lib, spec, status):
    letters = []
    for c in spec:
        if c.isalpha() and c not in letters:
            letters.append(c)
    if spec == "ijk,ja,ka->i a":
        p = dz.Plan(spec, [3] * len(letters))  # whitespace is ignored: this is MTTKRP mode 0
        assert p.kind == "mttkrp"
        return
    with pytest.raises(dz.DeinsumError) as e:
        dz.Plan(spec, [3] * len(letters))
    assert e.value.status == status


def test_plan_rejects_bad_extents_and_dtype(lib):
    with pytest.raises(dz.DeinsumError) as e:
        dz.Plan("ijk,ja,ka->ia", [3, 3, 3])        # one extent missing
    assert e.value.status == 3
    with pytest.raises(dz.DeinsumError) as e:
        dz.Plan("ijk,ja,ka->ia", [3, 0, 3, 4])     # zero extent
    assert e.value.status == 3
    with pytest.raises(dz.DeinsumError) as e:
        dz.Plan("ijk,ja,ka->ia", [3, 3, 3, 4], dtype="float64", prec="split_bf16")
    assert e.value.status == 4
    with pytest.raises(dz.DeinsumError) as e:
        dz.Plan("ijk,ja,ka->ia", [3, 3, 3, 65])    # rank above 64
    assert e.value.status == 2


def test_plan_info_counts(lib):
    p = dz.Plan("ijk,ja,ka->ia", [1024, 1024, 1024, 32])
    info = p.info()
    x = 1024 ** 3
    assert info["alg_flops"] == 2.0 * x * 32
    assert info["alg_bytes"] == 4.0 * (x + 3 * 1024 * 32)
    t = dz.Plan("ijkl,jb,kc,ld->ibcd", [256, 256, 256, 256, 32, 32, 32])
    ti = t.info()
    # FLOP-minimal chain: 2*256^4*32 + 2*256^3*32*32 + 2*256^2*32^3
    assert ti["alg_flops"] == 2.0 * (256 ** 4 * 32 + 256 ** 3 * 32 * 32 + 256 ** 2 * 32 ** 3)
    assert ti["out_elems"] == 256 * 32 ** 3


def test_status_strings(lib):
    for code in range(10):
        assert lib.deinsum_status_string(code)


def test_einsum_builders():
    assert dz.mttkrp_einsum(3, 0) == "abc,br,cr->ar"
    assert dz.mttkrp_einsum(5, 2) == "abcde,ar,br,dr,er->cr"
    assert dz.ttmc_einsum(4, 0) == "abcd,bt,cu,dv->atuv"


def test_split_ttmc_plan_rules(lib):
    """Split-BF16 TTMc is the fused last-two-mode kernel: kept mode below N-2,
    R_{N-2}, R_{N-1} <= 32 and I_{N-1} a multiple of 4; other shapes are refused
    at plan time (status 2) rather than silently run another way."""
    ok = dz.Plan(dz.ttmc_einsum(4, 0), [20, 30, 130, 64, 5, 16, 12], prec="split_bf16")
    assert ok.info()["kind"] == "ttmc"
    # rows of I_{N-1} = 66 words are not 16-byte aligned: the row-class maps take them
    dz.Plan(dz.ttmc_einsum(4, 0), [20, 30, 130, 66, 5, 16, 12], prec="split_bf16")
    dz.Plan(dz.ttmc_einsum(3, 0), [50, 300, 132, 17, 31], prec="split_bf16")
    dz.Plan(dz.ttmc_einsum(5, 2), [6, 7, 8, 90, 44, 4, 6, 9, 32], prec="split_bf16")
    for spec, ext in [
        (dz.ttmc_einsum(4, 3), [20, 30, 130, 64, 5, 16, 12]),   # kept mode N-1
        (dz.ttmc_einsum(4, 2), [20, 30, 130, 64, 5, 16, 12]),   # kept mode N-2
        (dz.ttmc_einsum(4, 0), [20, 30, 130, 64, 5, 16, 33]),   # R_{N-1} > 32
        (dz.ttmc_einsum(4, 0), [20, 30, 130, 64, 5, 40, 12]),   # R_{N-2} > 32
    ]:
        with pytest.raises(dz.DeinsumError) as e:
            dz.Plan(spec, ext, prec="split_bf16")
        assert e.value.status == 2, (spec, ext)
    # the plain precision takes every TTMc shape
    dz.Plan(dz.ttmc_einsum(4, 3), [20, 30, 130, 64, 5, 16, 12], prec="plain")


def test_graft_entry_imports():
    import importlib
    g = importlib.import_module("__graft_entry__")
    assert callable(g.build) and callable(g.smoke)


def test_mttkrp_mm_plan(lib):
    """MTTKRP + MM (Sec. II-A running example ijk,ja,ka,al->il): an extra trailing
    operand <rank><new letter> and output <kept><new letter>."""
    p = dz.Plan("ijk,ja,ka,al->il", [100, 30, 40, 24, 16])
    info = p.info()
    assert info["kind"] == "mttkrp" and info["mode"] == 0 and info["mm_cols"] == 16
    assert info["out_elems"] == 100 * 16
    x = 100 * 30 * 40
    assert info["alg_flops"] == 2.0 * x * 24 + 2.0 * 100 * 24 * 16
    assert info["alg_bytes"] == 4.0 * (x + 30 * 24 + 40 * 24 + 24 * 16 + 100 * 16)
    assert dz.mttkrp_mm_einsum(3, 0) == "abc,br,cr,rl->al"
    dz.Plan(dz.mttkrp_mm_einsum(4, 3), [5, 6, 7, 8, 9, 10], prec="split_bf16")
    for spec in ["ijk,ja,ka,ak->il",     # C's second letter is a letter of X
                 "ijk,ja,ka,bl->il",     # C does not start with the rank letter
                 "ijk,ja,ka,al->ia",     # output keeps the rank letter
                 "ijk,ja,kb,al->il"]:    # factors do not share one rank letter
        with pytest.raises(dz.DeinsumError) as e:
            letters = []
            for c in spec.replace(",", "").replace("->", ""):
                if c not in letters:
                    letters.append(c)
            dz.Plan(spec, [4] * len(letters))
        assert e.value.status == 2, spec


def test_mttkrp_row_view_decisions(lib):
    """The planner's row view: merged short inner modes, packed outer indices for short
    rows, leading indices per tile (at most 16), and how X's rows are loaded (one tensor
    map when the rows are 16-byte aligned, else the four row-class maps)."""
    def view(dims, mode, prec="split_bf16", R=8):
        return dz.Plan(dz.mttkrp_einsum(len(dims), mode), list(dims) + [R], "float32", prec).info()["view"]

    for mode in range(3):   # 1024^3: aligned rows, no regrouping
        assert view((1024, 1024, 1024), mode) == {"merged": False, "packed": False, "groups": 1,
                                                  "aligned_rows": True, "row_classes": False}
        v = view((1023, 1023, 1023), mode)
        assert not v["aligned_rows"] and v["row_classes"]
    # inner mode of 47 merged with its neighbour of 5: mode 0 then packs 14 outer indices of
    # 9 rows; mode 1 takes 8 leading indices of 15 rows; mode 2 (not merged: its inner mode is
    # the last one) is capped at 16 leading indices of 5 rows; the last mode packs again
    assert view((9, 15, 5, 47), 0) == {"merged": True, "packed": True, "groups": 14,
                                       "aligned_rows": False, "row_classes": False}
    assert view((9, 15, 5, 47), 1) == {"merged": True, "packed": False, "groups": 8,
                                       "aligned_rows": False, "row_classes": True}
    assert view((9, 15, 5, 47), 2)["groups"] == 16 and not view((9, 15, 5, 47), 2)["merged"]
    assert view((9, 15, 5, 47), 3)["packed"]
    # a last mode of 77 rows is not packed (rows above 64) and takes the row classes
    v = view((3, 301, 77), 2)
    assert not v["packed"] and v["row_classes"]
    assert view((40, 6, 7, 8, 36), 0)["packed"] and view((40, 6, 7, 8, 36), 0)["groups"] == 3
    # the plain precision neither merges nor uses row classes
    v = view((9, 15, 5, 47), 1, prec="plain")
    assert not v["merged"] and not v["row_classes"]
    # TTMc plans carry no MTTKRP view
    assert dz.Plan(dz.ttmc_einsum(3, 0), [50, 300, 132, 17, 31], prec="split_bf16").info()["view"]["groups"] == 0
