"""Host-side helpers of bench.py (CPU): the kernel-source hash that keys the
committed ncu counters ignores comments and layout but not code."""
import bench


def test_strip_comments_keeps_code_and_literals():
    src = 'int a = 1; // note\n/* block\n comment */ const char* s = "// not a comment";\n'
    assert bench._strip_comments(src) == 'int a = 1; const char* s = "// not a comment";'


def test_hash_input_ignores_comments_only():
    a = "__global__ void k(int* p) {\n    p[0] = 1;   // store\n}\n"
    b = "/* header */\n__global__ void k(int* p) { p[0] = 1; }\n"
    c = "__global__ void k(int* p) { p[0] = 2; }\n"
    assert bench._strip_comments(a) == bench._strip_comments(b)
    assert bench._strip_comments(a) != bench._strip_comments(c)
