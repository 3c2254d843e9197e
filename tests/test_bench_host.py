"""Host-side logic of bench.py: the coarse-tail flag and the key that ties a recorded
DRAM traffic figure to the code of the kernel it was measured on."""
import argparse
import os

import bench

SWEEP = os.path.join(os.path.dirname(__file__), "..", "paper_1609_04809_gb300", "csrc", "sweep.cuh")


def test_tail_mode():
    ns = lambda **kw: argparse.Namespace(**{"no_tail": False, "tail": "auto", **kw})  # noqa: E731
    assert bench._tail_mode(ns()) == 2
    assert bench._tail_mode(ns(tail="on")) == 1
    assert bench._tail_mode(ns(tail="off")) == 0
    assert bench._tail_mode(ns(no_tail=True, tail="on")) == 0


def test_storage_names_round_trip():
    for name, code in bench.STORAGES.items():
        assert bench.STORAGE_NAMES[code] == name


def test_kernel_key_follows_the_kernel_code_only():
    src = open(SWEEP).read()
    key = bench._kernel_sha("dia", src)
    assert key == bench._kernel_sha("dia")
    # comments and blank lines do not change it
    commented = src.replace("__global__ void __launch_bounds__(256) k_dia_sweep",
                            "// a remark\n\n__global__ void __launch_bounds__(256) k_dia_sweep", 1)
    assert commented != src and bench._kernel_sha("dia", commented) == key
    # code after the kernel (another kernel) does not change it
    later = src.replace("struct StencilView {", "struct StencilView {\n    int unused;", 1)
    assert later != src and bench._kernel_sha("dia", later) == key
    # a change inside the kernel does
    changed = src.replace("if (i >= n) return;\n    constexpr int C = K / 2;",
                          "if (i >= n) return;\n    constexpr int C = K / 2 + 0;", 1)
    assert changed != src and bench._kernel_sha("dia", changed) != key
    # every storage with a sweep kernel has a key
    assert len({bench._kernel_sha(st, src) for st in bench.SWEEP_KERNELS}) == len(bench.SWEEP_KERNELS)
