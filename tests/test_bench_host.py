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


def test_launch_count_of_whole_loop_bodies():
    # 17 loop passes: three bodies of 8 in graph mode (24 passes launched, the
    # last 7 returning at once), one chunk of 32 in the chunked mode
    rr = [{"iterations": 17, "force_evals": 18, "nbr_builds": 2}]
    setup = 1 + 6 + 3 + 1 + 1
    graph = bench.launches_of(rr, is_rgl=True, fp32=False, cell_mode=True)
    assert graph == setup + 5 * 24 + 6 * 1       # one rebuild under its IF node
    chunked = bench.launches_of(rr, is_rgl=True, fp32=False, cell_mode=True, chunked=True)
    assert chunked == setup + 5 * 32 + 6 * 32    # gated build chain every pass
    allpairs = bench.launches_of(rr, is_rgl=False, fp32=False, cell_mode=False)
    assert allpairs == (1 + 1 + 1 + 1 + 1) + 3 * 24 + 1 * 24
