"""Host logic of bench.py that decides whether the recorded ncu counters still
describe the kernels: the hash covers the code of the kernel sources, not
their comments or layout."""

import bench


def test_code_only_drops_comments_and_layout():
    src = "int a = 1;  // one\n/* block\n comment */ int b =\n    2; // two\n"
    assert bench.code_only(src) == "int a = 1; int b = 2;"


def test_kernel_hash_follows_code_not_comments():
    files = {"common.cuh": "int f() { return 1; }\n", "kernels.cuh": "// k\nint g();\n",
             "pipeline.cuh": "int h();\n"}
    base = bench.kernel_hash(files.__getitem__)
    commented = dict(files, **{"kernels.cuh": "/* kernels */\nint   g();  // declared here\n"})
    assert bench.kernel_hash(commented.__getitem__) == base
    changed = dict(files, **{"kernels.cuh": "int g(int);\n"})
    assert bench.kernel_hash(changed.__getitem__) != base


def test_kernel_hash_reads_the_working_tree():
    h = bench.kernel_hash()
    assert len(h) == 16 and int(h, 16) >= 0
