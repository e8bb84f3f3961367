"""Host logic of bench.py (no GPU): the algorithmic HBM byte model behind
the roofline fractions, and the workload table.

The byte model counts, per transform, each point record (index, packed cell,
d offsets) and value once per pass, the oversampled grid once per pass, two
passes per FFT, and I_N once per scaling pass.  The per-stage model of the 3-D
configuration and the generic per-transform model must agree, and the terms
are checked by hand for a small case."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_stage_model_equals_transform_model(bench):
    wl = bench.WORKLOADS["config"]
    per_set = sum(bench._stage_hbm_bytes(s, wl["N"], wl["M"]) for s in ("sort", "spread", "fft", "deconv", "pad",
                                                                         "ifft", "interp"))
    assert per_set == bench._transform_bytes(wl["N"], wl["M"])


def test_stage_model_of_the_3d_configuration(bench):
    # N = 64^3, n = 128^3, M = 1e6, complex64: the spreading launch moves each
    # point's three FP32 offsets and its value (20 B) and the grid once (8 B
    # per cell): 36.8 MB
    N, M, cells = (64, 64, 64), 10 ** 6, 128 ** 3
    assert bench._stage_hbm_bytes("spread", N, M) == M * 20 + cells * 8 == 36777216
    assert bench._stage_hbm_bytes("sort", N, M) == M * (24 + 8 + 12)
    # the picker may take sigma = 1.5: n = 384 (2^7 x 3)
    assert bench._cells((256, 256, 256), 1.5) == 384 ** 3
    assert bench._cells((100,), 1.25) == 126


def test_transform_model_by_hand(bench):
    # 1-D, N = 8, n = 16, M = 3, FP64: offsets 8 B, value 16 B, cell 16 B
    N, M, cells, NN = (8,), 3, 16, 8
    rec, cz = 8, 16
    sort = M * (8 + 8 + rec)
    adjoint = M * (rec + cz) + cells * cz + 2 * cells * cz + NN * cz * 2
    forward = (cells + NN) * cz + 2 * cells * cz + M * (rec + cz) + cells * cz
    assert bench._transform_bytes(N, M, 2.0, 1, 8) == sort + adjoint + forward
    assert bench._transform_bytes(N, M, 2.0, 1, 8, sort=False, forward=False) == adjoint
    # an Ewald adjoint reads its weighted modes once instead of writing fhat
    ewald = M * (rec + cz) + cells * cz + 2 * cells * cz + NN * cz
    assert bench._transform_bytes(N, M, 2.0, 1, 8, sort=False, forward=False, ewald=True) == ewald
    # right-hand sides multiply values, grids and modes, not the point records
    r2 = bench._transform_bytes(N, M, 2.0, 2, 8, sort=False, forward=False)
    assert r2 == M * (rec + 2 * cz) + 2 * (cells * cz + 2 * cells * cz + NN * cz * 2)


def test_workload_table(bench):
    for name, wl in bench.WORKLOADS.items():
        assert wl["name"] and wl["sets"], name
        if name != "batch":
            assert len(wl["N"]) in (1, 3) and wl["M"] > 0, name
    assert bench.WORKLOADS["fig16"]["M"] == 12 * bench.WORKLOADS["fig16"]["lc"] ** 3
    assert bench.WORKLOADS["fig13"]["M"] == 120 ** 3
    # the default line runs the largest configuration
    big = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    assert big["N"] == (256, 256, 256) and big["M"] == 30_000_000 and big["eps"] == 1e-5
