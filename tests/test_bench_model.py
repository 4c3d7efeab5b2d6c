"""The benchmark's per-phase work model and roofline arithmetic (bench.py),
checked against values worked out by hand (no GPU).

Pass model: every FP32 or tensor-core pass reads and writes the tensor once
(complex64: 16 B per entry, +8 B where it reads or writes complex128, +16 B for
the correction's last back pass, which also reads X); the sweep moves 16 B per
entry and solve; a tensor-core residual pass 48 B.  FP64 phases count flops:
the method's 8 n_j per entry and mode, and the executed 6 n_j where the
three-multiplication product runs (residual always, transforms for even
n_j >= 8)."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402

E = 64 ** 4


def desc(P, residual_passes=4, residual_tc=0, diag=0):
    return {"transform_passes": P, "residual_passes": residual_passes,
            "residual_tc": residual_tc, "diag_sweep": diag}


def test_mixed_pass_model_64_4():
    w = bench.phase_work("mixed", desc(4), (64,) * 4, E, 1)
    # forward: first transform reads c128 B (4 passes x 16 B + 8 B), the
    # correction's transform reads the c128 residual (+8 B)
    assert w["forward"] == ("hbm", (72 + 72) * E, None)
    # back: the solve's last pass writes c128 X (+8 B); the correction's last
    # pass reads and writes X (+24 B)
    assert w["back"] == ("hbm", (72 + 88) * E, None)
    assert w["sweep"] == ("hbm", 32 * E, None)          # two sweeps, 16 B each
    # FP64 residual, one refinement step: method 8 x 256 flops per entry,
    # executed 6 x 256
    assert w["residual"] == ("fp64", 2048 * E, 1536 * E)


def test_tensor_core_residual_pass_model():
    w = bench.phase_work("mixed_emu", desc(4, residual_passes=4, residual_tc=1), (64,) * 4, E, 1)
    assert w["residual"] == ("hbm", 4 * 48 * E, None)
    # the tensor-core residual writes complex64 R straight into the working
    # tensor: the correction's forward transform reads no complex128
    assert w["forward"] == ("hbm", (72 + 64) * E, None)


def test_fp64_flop_counts_odd_and_even_modes():
    shape = (19, 64, 2, 1)
    En = 19 * 64 * 2
    w = bench.phase_work("fp64", desc(3), shape, En, 0)
    meth = 8 * (19 + 64 + 2) * En
    # executed: classical 8 n for odd n and n < 8, three multiplications for 64
    exe = (8 * 19 + 6 * 64 + 8 * 2) * En
    assert w["forward"] == ("fp64", meth, exe)
    assert w["back"] == ("fp64", meth, exe)
    # sweep: 4 sum_j (n_j - 1) + 11 flops per entry (the singleton adds 0)
    assert w["sweep"] == ("fp64", (4 * (18 + 63 + 1 + 0) + 11) * En,
                          (4 * (18 + 63 + 1 + 0) + 11) * En)
    # normal operators: the sweep is an entrywise division, 32 B per entry
    w = bench.phase_work("fp64", desc(3, diag=1), shape, En, 0)
    assert w["sweep"] == ("hbm", 32 * En, None)


def test_roofline_fractions():
    d = desc(4)
    phases = {"forward": 1.0, "back": 2.0, "sweep": 4.0, "residual": 10.0}
    out = bench.phase_roofline("mixed", phases, [d], [(64,) * 4], [E], 1, 8000.0)
    fwd_gbs = 144 * E / 1e-3 / 1e9
    assert out["forward"]["achieved_gbs"] == pytest.approx(fwd_gbs)
    assert out["forward"]["frac"] == pytest.approx(fwd_gbs / 8000.0)
    assert out["sweep"]["frac"] == pytest.approx(32 * E / 4e-3 / 1e9 / 8000.0)
    tf = 1536 * E / 10e-3 / 1e12
    assert out["residual"]["achieved_tflops"] == pytest.approx(tf)
    assert out["residual"]["frac"] == pytest.approx(tf / bench.FP64_PEAK_TFLOPS)
    assert out["residual"]["frac_method_count"] == pytest.approx(
        2048 * E / 10e-3 / 1e12 / bench.FP64_PEAK_TFLOPS)
    # phases not timed are left out; two equations add up
    out2 = bench.phase_roofline("mixed", {"sweep": 4.0}, [d, d], [(64,) * 4] * 2, [E, E], 1,
                                8000.0)
    assert set(out2) == {"sweep"}
    assert out2["sweep"]["frac"] == pytest.approx(2 * out["sweep"]["frac"])


def test_fp64_peak_and_traffic_key():
    # 152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.25856)
    sha = bench.kernels_sha()
    assert len(sha) == 16 and all(c in "0123456789abcdef" for c in sha)
    assert set(bench.TRAFFIC) >= {"kernels_sha", "bytes_per_launch", "source"}
