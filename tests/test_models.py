"""The paper's traffic and cache models (Sec. III) and their GPU counterparts.

Golden values: tests/golden/paper_numbers.json (printed in the paper).
"""
import json
import os

import pytest

from paper_1510_05218_gb300 import tuning

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def test_code_balance_models_match_the_paper():
    assert tuning.code_balance_naive() == GOLDEN["code_balance_naive"]
    assert tuning.code_balance_spatial() == GOLDEN["code_balance_spatial"]
    assert round(GOLDEN["flops_per_lup"] / tuning.code_balance_naive(), 2) == GOLDEN["intensity_naive"]
    assert round(GOLDEN["flops_per_lup"] / tuning.code_balance_spatial(), 2) == GOLDEN["intensity_spatial"]
    assert round(tuning.bottleneck_mlups(GOLDEN["bottleneck_bandwidth_gbs"], tuning.code_balance_spatial())) \
        == GOLDEN["bottleneck_mlups"]


def test_cache_block_model_worked_example_and_haswell_cases():
    ex = GOLDEN["cache_block_example"]
    assert tuning.cache_block_bytes(1, ex["D_w"], ex["B_Z"]) == ex["bytes_per_nx"]
    assert ex["D_w"] + ex["B_Z"] - 1 == ex["W_w"]
    # B_Z = 6, D_w = 4 with three thread groups (three tiles): "30 MiB";
    # B_Z = 1, D_w = 8 with two thread groups of nine threads: "20 MiB" (both approximate)
    c1 = 3 * tuning.cache_block_bytes(480, 4, 6) / 2 ** 20
    c2 = 2 * tuning.cache_block_bytes(480, 8, 1) / 2 ** 20
    assert abs(c1 - 30) <= 0.1 * 30 and abs(c2 - 20) <= 0.1 * 20
    assert c2 > GOLDEN["usable_l3_mib"] * 0.9 and c1 > GOLDEN["usable_l3_mib"]


def test_diamond_code_balance_decreases_with_width():
    vals = [tuning.code_balance_diamond(d) for d in (4, 8, 12, 16)]
    assert [round(v) for v in vals] == [428, 211, 140, 105]
    assert vals[1] < tuning.code_balance_spatial() / 5      # "6x lower code balance" regime


@pytest.mark.parametrize("precision,temporal", [(0, 1), (1, 1), (2, 1), (1, 2)])
def test_gpu_footprint_and_balance(precision, temporal):
    fp = tuning.gpu_footprint(precision, temporal, 64, 8192, 152, 129 * 2 ** 20)
    assert fp["smem_per_cta"] <= tuning.SMEM_PER_CTA and fp["fits"]
    b = tuning.gpu_code_balance(precision, temporal, 64)
    alg = 52 * tuning.elem_bytes(precision)
    if temporal == 1:
        assert alg < b < 1.3 * alg            # the halo re-read of the tiles: +10..30 %
    else:
        assert b < 0.75 * alg                 # two iterations per pass: fewer bytes per iteration


def test_candidates_respect_the_model():
    c = tuning.candidates(1, 512, 1024, 152, 129 * 2 ** 20)
    assert (1, 64) in c and any(t == 2 for t, _ in c)
    assert all(t == 1 for t, _ in tuning.candidates(0, 512, 1024, 152, 129 * 2 ** 20))


def test_footprint_model_matches_the_kernels_shared_memory():
    """The footprint model's shared memory per CTA equals what ptxas reports for
    the sweep kernels (plus the 2 x NT/32 doubles of the norm reduction)."""
    import concurrent.futures as cf
    import re
    import shutil
    import subprocess

    from paper_1510_05218_gb300 import build

    nvcc = build._nvcc()
    if shutil.which(nvcc) is None and not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    # (source, precision, iterations per launch, threads, grid cells); the
    # FP64 sweep runs 32 x 16 tiles on large grids and 32 x 8 below 2^23 cells
    cases = [("thiim_sweep_f64.cu", 0, 1, 256, None), ("thiim_noalloc.cu", 0, 1, 256, 64 ** 3),
             ("thiim_sweep_f32.cu", 1, 1, 256, None), ("thiim_sweep_pair_b.cu", 2, 1, 256, None),
             ("thiim_sweep2_f32.cu", 1, 2, 512, None)]

    def smem(src):
        cmd = [nvcc, *build.ARCH, "-O3", "-std=c++17", "-I", build.INCLUDE, "-I", build.CSRC, "-Xptxas", "-v",
               "-cubin", "-o", os.devnull, os.path.join(build.CSRC, src)]
        out = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
        assert out.returncode == 0, out.stderr[-2000:]
        return {int(v) for v in re.findall(r"(\d+) bytes smem", out.stderr)}

    with cf.ThreadPoolExecutor(4) as ex:
        found = list(ex.map(lambda c: smem(c[0]), cases))
    for (src, precision, temporal, nt, cells), sizes in zip(cases, found):
        model = tuning.gpu_footprint(precision, temporal, 32, 8192, 152, 129 * 2 ** 20, cells)["smem_per_cta"]
        # the file's plain sweep (a second kernel there, e.g. the defect sweep, may differ)
        assert model + 2 * (nt // 32) * 8 in sizes, (src, sizes, model)


def test_fp64_tile_rule_matches_the_library():
    """tuning.tile's FP64 size rule (32 x 16 from F64_TALL_MIN_CELLS cells on,
    32 x 8 below) is the library's: the threshold and both tile heights are
    read from the CUDA headers."""
    import re

    from paper_1510_05218_gb300 import build

    src = open(os.path.join(build.CSRC, "thiim_internal.h")).read()
    m = re.search(r"#define THIIM_F64_TALL_MIN_CELLS \(1ull << (\d+)\)", src)
    assert m and tuning.F64_TALL_MIN_CELLS == 1 << int(m.group(1))
    tall_ty = int(re.search(r"#define THIIM_SWEEP_F64_TY (\d+)", src).group(1))
    short_ty = int(re.search(r"#define THIIM_SWEEP_TY (\d+)", src).group(1))
    n = tuning.F64_TALL_MIN_CELLS
    assert tuning.tile(0, n) == (tuning.TX, tall_ty)
    assert tuning.tile(0, n - 1) == (tuning.TX, short_ty)
    assert tuning.tile(0) == (tuning.TX, tall_ty)            # size unknown: the large-grid tile
    assert tuning.tile(1, 64 ** 3) == tuning.tile(1) == (tuning.TX, tuning.TY)
    # the footprint model follows: 3 CTAs/SM on the short FP64 tile, 2 on the tall one
    assert tuning.gpu_footprint(0, 1, 32, 8192, 152, 129 * 2 ** 20, n - 1)["ctas_per_sm"] == 3
    assert tuning.gpu_footprint(0, 1, 32, 8192, 152, 129 * 2 ** 20, n)["ctas_per_sm"] == 2
