"""The plan-time code generators (CPU): sources written for representative shapes (the
Retailer- and Favorita-like lean passes, a pass without an inner relation, a decision-tree
level with leaf bits, leaf histograms, leaf-split partials and per-leaf CTA-private bucket
items, and a general pass with an indicator factor and CTA-private items grouped by root
buckets) compile with NVRTC for sm_103a, in FP32 and FP64, without register
spills. Needs nvcc and NVRTC, not a GPU."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


@pytest.fixture(scope="module")
def results():
    if not os.path.exists(NVCC):
        pytest.skip("nvcc is not installed")
    tmp = tempfile.mkdtemp()
    try:
        exe = os.path.join(tmp, "codegen_check")
        csrc = os.path.join(ROOT, "paper_2008_08657_b300", "csrc")
        lib = os.path.join(os.path.dirname(os.path.dirname(NVCC)), "lib64")
        subprocess.run([NVCC, "-std=c++17", "-I", os.path.join(ROOT, "include"), "-o", exe,
                        os.path.join(ROOT, "tests", "codegen_check.cu"), os.path.join(csrc, "codegen.cpp"),
                        os.path.join(csrc, "codegen_family.cpp"), "-L" + lib, "-lnvrtc", "-Xlinker", "-rpath=" + lib],
                       check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    return {line.split()[0]: line.split()[1:] for line in out.splitlines() if line.strip()}


SHAPES = ["view_weather", "view_item"] + [f"{s}_{p}" for s in ("lean_retailer", "lean_retailer_lanes", "lean_favorita", "lean_no_inner", "dt_level", "dt_leaf_sums",
                                    "general_no_inner")
          for p in ("fp32", "fp64")]


@pytest.mark.parametrize("shape", SHAPES)
def test_generated_source_compiles_without_spills(results, shape):
    assert shape in results, results
    status = results[shape]
    assert status[0] == "ok", " ".join(status)
    regs, spill = int(status[1]), int(status[2])
    # root passes run 1024 threads per SM (64 registers each in FP32); view kernels 128-thread CTAs
    assert 0 < regs <= (128 if shape.endswith("fp64") or shape.startswith("view") else 64)
    assert spill == 0
