"""Host-side helpers of bench.py, on the CPU: the code-only view behind the traffic records.

A committed ncu traffic record stays current while the code of the files its kernel is
compiled from is unchanged; comments may change.  `_code_only` must therefore drop every
comment and blank line, keep string and character literals whole (a "//" inside one is
code), and change whenever a token of code changes.
"""
import bench


def test_comments_and_blank_lines_dropped():
    src = "int a = 1; // one\n\n/* two\n   lines */ int b = 2;\n   int c;  \n"
    assert bench._code_only(src) == "int a = 1;\nint b = 2;\nint c;"


def test_literals_kept_whole():
    src = 'asm("cp.async.bulk [%0]; // not a comment");\nchar q = \'"\'; char s = \'/\';\n'
    out = bench._code_only(src)
    assert '"cp.async.bulk [%0]; // not a comment"' in out
    assert "char q = '\"';" in out and "char s = '/';" in out


def test_escaped_quote_inside_string():
    src = 'const char *s = "a\\"b // c"; int x; // tail\n'
    assert bench._code_only(src) == 'const char *s = "a\\"b // c"; int x;'


def test_comment_edits_keep_the_view_and_code_edits_change_it():
    a = "__global__ void k(float *x) {\n    x[0] = 1.f;   // store\n}\n"
    b = "// a new header comment\n__global__ void k(float *x) {\n    /* reworded */ x[0] = 1.f;\n}\n"
    c = "__global__ void k(float *x) {\n    x[1] = 1.f;   // store\n}\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)

