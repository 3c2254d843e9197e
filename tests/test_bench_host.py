"""Host-side logic of bench.py: the coarse-tail flag, workload scaling for profiling, and
the key that ties a recorded DRAM traffic figure to the code of the kernel it was
measured on."""
import argparse
import os

import bench

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_1609_04809_gb300", "csrc")


def _sources():
    return {f: open(os.path.join(CSRC, f)).read() for f in ("sweep.cuh", "kernels.cuh")}


def test_tail_mode():
    ns = lambda **kw: argparse.Namespace(**{"no_tail": False, "tail": "auto", **kw})  # noqa: E731
    assert bench._tail_mode(ns()) == 2
    assert bench._tail_mode(ns(tail="on")) == 1
    assert bench._tail_mode(ns(tail="off")) == 0
    assert bench._tail_mode(ns(no_tail=True, tail="on")) == 0


def test_storage_names_round_trip():
    for name, code in bench.STORAGES.items():
        assert bench.STORAGE_NAMES[code] == name


def test_smaller_case_keeps_the_coarsest_grid():
    c = bench._config_args("q1_3d_256_vark", cells=128)
    assert c["n_cells"] == 128 and c["n_levels"] == 6 and c["precision"] == "mixed"
    assert bench._config_args("q1_3d_256_vark")["n_levels"] == 7


def test_kernel_key_follows_the_kernel_code_only():
    src = _sources()
    for kernel in bench.KERNEL_PARTS:
        key = bench._kernel_sha(kernel, src)
        assert key == bench._kernel_sha(kernel)
    key = bench._kernel_sha("k_dia_sweep", src)
    sweep = src["sweep.cuh"]
    # comments and blank lines do not change it
    commented = sweep.replace("template <typename T, int K, int MODE>\n__global__ void __launch_bounds__(256) k_dia_sweep",
                              "// a remark\n\ntemplate <typename T, int K, int MODE>\n"
                              "__global__ void __launch_bounds__(256) k_dia_sweep", 1)
    commented = commented.replace("    if (i >= n) return;\n    constexpr int C = K / 2;",
                                  "    if (i >= n) return;  // past the end\n\n    constexpr int C = K / 2;", 1)
    assert commented != sweep and bench._kernel_sha("k_dia_sweep", {**src, "sweep.cuh": commented}) == key
    # code outside the kernel's parts (another kernel) does not change it
    later = sweep.replace("struct StencilView {", "struct StencilView {\n    int unused;", 1)
    assert later != sweep and bench._kernel_sha("k_dia_sweep", {**src, "sweep.cuh": later}) == key
    # a change inside the kernel, or in a helper it calls, does
    changed = sweep.replace("if (i >= n) return;\n    constexpr int C = K / 2;",
                            "if (i >= n) return;\n    constexpr int C = K / 2 + 0;", 1)
    assert changed != sweep and bench._kernel_sha("k_dia_sweep", {**src, "sweep.cuh": changed}) != key
    helper = sweep.replace("o = A::sub(bi, s);", "o = A::sub(bi, s) + T(0);", 1)
    assert helper != sweep and bench._kernel_sha("k_dia_sweep", {**src, "sweep.cuh": helper}) != key
    # the outer residual's key follows kernels.cuh's reduction helpers
    k = src["kernels.cuh"]
    red = k.replace("constexpr int kReduceBlocks = 912;", "constexpr int kReduceBlocks = 912; // same", 1)
    assert bench._kernel_sha("k_outer_resid", {**src, "kernels.cuh": red}) == bench._kernel_sha("k_outer_resid", src)
    fin = k.replace("*ticket = 0u;", "*ticket = 0u + 0u;", 1)
    assert fin != k and bench._kernel_sha("k_outer_resid", {**src, "kernels.cuh": fin}) != bench._kernel_sha(
        "k_outer_resid", src)
    # and its residency (a one-line function in its launch bounds)
    occ = k.replace("return fmt == 3 ? 3 : 6;", "return fmt == 3 ? 4 : 6;", 1)
    assert occ != k and bench._kernel_sha("k_outer_resid", {**src, "kernels.cuh": occ}) != bench._kernel_sha(
        "k_outer_resid", src)
    one = bench._source_part(k, "fp64_rows_blocks_per_sm")
    assert one.startswith("constexpr int fp64_rows_blocks_per_sm(") and one.count("\n") == 1
