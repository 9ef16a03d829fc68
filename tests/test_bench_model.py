"""Host logic of the benchmark: the launch and byte model of one sketched reconstruction on the
large cones workload against the counts of the ncu launch list of the same command (spread and
interpolation 280 launches each, strided passes 960, x passes 240 each, for T = 20 outer
iterations of K = 10 with m = 10 sketched coils), and the
NUFFT byte models against their closed forms."""
import bench


def test_launch_model_matches_the_measured_launch_list():
    w = dict(bench.WORKLOAD)
    T = 20
    expect = {"spread": 280, "interp": 280, "fft_plain": 960, "expand": 240, "reduce": 240}
    for stage, n in expect.items():
        _, launches = bench.stage_bytes(stage, w, T, 10, 10, 1)
        assert launches == n, stage
    b1, _ = bench.stage_bytes("spread", w, T, 10, 10, 1)
    b3, _ = bench.stage_bytes("spread", w, T, 10, 10, 3)
    assert b3 == 3 * b1


def test_nufft_byte_models():
    w = dict(bench.WORKLOAD)
    D, G, N, C = 160 * 256 * 256, 200 * 320 * 320, 20000 * 512, 40
    assert bench.nufft_model_bytes(w, C) == 2 * C * (8 * D + 48 * G + 8 * N) + 2 * (16 * N + 16 * D)
    assert bench.nufft_compulsory_bytes(w, C) == C * (8 * D + 8 * N) * 2 + 16 * N + 16 * D
    assert 92.5e9 < bench.nufft_model_bytes(w, C) < 92.6e9
    assert 13.5e9 < bench.nufft_compulsory_bytes(w, C) < 13.7e9
