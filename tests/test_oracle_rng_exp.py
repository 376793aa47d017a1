"""Pins for the oracle's Philox4x32-10 and its exp / threshold helpers.

Philox is checked against an independent third-party implementation (Triton's
philox_impl, run by Triton's CPU interpreter on numpy); mc_exp32 against the
C library's FP64 exp.
"""
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from oracle import oracle as orc

TRITON_SCRIPT = textwrap.dedent(r"""
    import os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(out_ptr, c_ptr, k_ptr, n: tl.constexpr):
        o = tl.arange(0, n)
        u = tl.uint32
        c0 = tl.load(c_ptr + 4 * o).to(u, bitcast=True)
        c1 = tl.load(c_ptr + 4 * o + 1).to(u, bitcast=True)
        c2 = tl.load(c_ptr + 4 * o + 2).to(u, bitcast=True)
        c3 = tl.load(c_ptr + 4 * o + 3).to(u, bitcast=True)
        k0 = tl.load(k_ptr + 2 * o).to(u, bitcast=True)
        k1 = tl.load(k_ptr + 2 * o + 1).to(u, bitcast=True)
        a, b, c, d = tl.philox_impl(c0, c1, c2, c3, k0, k1, 10)
        tl.store(out_ptr + 4 * o, a.to(tl.int32, bitcast=True))
        tl.store(out_ptr + 4 * o + 1, b.to(tl.int32, bitcast=True))
        tl.store(out_ptr + 4 * o + 2, c.to(tl.int32, bitcast=True))
        tl.store(out_ptr + 4 * o + 3, d.to(tl.int32, bitcast=True))

    data = np.load(sys.argv[1])
    n = data["ctr"].shape[0]
    ctr = torch.from_numpy(data["ctr"].view(np.int32).reshape(-1).copy())
    key = torch.from_numpy(data["key"].view(np.int32).reshape(-1).copy())
    out = torch.zeros(4 * n, dtype=torch.int32)
    k[(1,)](out, ctr, key, n)
    np.save(sys.argv[2], out.numpy().view(np.uint32).reshape(n, 4))
""")


def test_philox_matches_independent_implementation(tmp_path):
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    n = 256
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 0xFFFFFFFF
    key[1] = 0xFFFFFFFF
    np.savez(tmp_path / "in.npz", ctr=ctr, key=key)
    script = tmp_path / "tri.py"
    script.write_text(TRITON_SCRIPT)
    env = dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES="")
    subprocess.check_call([sys.executable, str(script), str(tmp_path / "in.npz"),
                           str(tmp_path / "out.npy")], env=env, timeout=600)
    ref = np.load(tmp_path / "out.npy")
    mine = np.stack([orc.philox(key[i], ctr[i]) for i in range(n)])
    np.testing.assert_array_equal(mine, ref)


def test_philox_uniformity_and_counter_sensitivity():
    # chi-square over the 256 byte values of 20000 words, and avalanche on one counter bit
    words = np.concatenate([orc.philox([11, 22], [i, 0, 0, 0]) for i in range(5000)])
    counts = np.bincount((words & 0xFF).astype(np.int64), minlength=256)
    expected = words.size / 256
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 256 + 6 * math.sqrt(2 * 256)
    a = orc.philox([1, 2], [3, 4, 5, 6])
    b = orc.philox([1, 2], [3 ^ 1, 4, 5, 6])
    flipped = sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b))
    assert 32 < flipped < 96


def test_taylor_coefficients_are_float_reciprocal_factorials():
    # the polynomial constants of the frozen exp are the FP32 roundings of 1/k!
    src = open(orc.SRC_PATH).read()
    for k in (7, 6, 5, 4):
        assert f"1.0f / {math.factorial(k)}.0f" in src
    assert np.float32(1.0) / np.float32(5040.0) == np.float32(1.0 / 5040.0)


def test_mc_exp32_error_bound():
    xs = np.concatenate([np.linspace(-64.0, 0.0, 20001, dtype=np.float32),
                         -np.logspace(-8, 0, 200).astype(np.float32)])
    worst = 0.0
    for x in xs:
        got = orc.mc_exp32(float(x))
        ref = math.exp(float(x))
        worst = max(worst, abs(got - ref) / ref)
    # degree-7 Taylor at |r| <= ln2/2 plus FP32 rounding: a few ulp
    assert worst < 4.0 * 2.0 ** -23, worst
    assert orc.mc_exp32(0.0) == 1.0


def test_t32_threshold_properties():
    assert orc.t32(0.0) == 0xFFFFFFFF
    assert orc.t32(-64.5) == 0
    assert orc.t32(-30.0) == 0  # e^-30 * 2^32 < 1
    prev = 0xFFFFFFFF
    for x in np.linspace(-0.0001, -22.0, 3001):
        v = orc.t32(float(np.float32(x)))
        assert v <= prev
        prev = v
        ref = math.exp(float(np.float32(x))) * 2.0 ** 32
        assert abs(v - ref) <= max(2.0, ref * 5e-7)


def test_screen_guard_band_absorbs_the_approximation_errors():
    """The Gaussian sweep screens r <= T32(x) by the sign of fl(r) - A, with
    A ~ e^x 2^32 from a fast 2^x, deciding only outside |fl(r) - A| <= 2^-12 A
    (the device test checks the hardware). Here A is e^x 2^32 moved by a
    relative error of +-2^-16, four times the bound the design states, and
    every decision the screen would take outside the band must equal the
    oracle's r <= T32(x) at and around each threshold and on random draws."""
    rng = np.random.default_rng(5)
    xs = np.concatenate([np.linspace(-64.0, 0.0, 4001, dtype=np.float32),
                         -(rng.random(2000) * 23).astype(np.float32)])
    band = 2.0 ** -12
    decided = 0
    for x in xs:
        thr = orc.t32(float(x)) if x < 0 else 0xFFFFFFFF
        exact = math.exp(float(x)) * 2.0 ** 32
        rs = {thr, max(thr - 1, 0), min(thr + 1, 2 ** 32 - 1), min(thr + 2, 2 ** 32 - 1),
              int(rng.integers(0, 2 ** 32)), 0, 2 ** 32 - 1}
        for eps in (-2.0 ** -16, 2.0 ** -16):
            a = float(np.float32(exact * (1.0 + eps)))
            for r in rs:
                fr = float(np.float32(r))
                u = float(np.float32(fr - a))
                if abs(u) > band * a:
                    decided += 1
                    assert (u < 0) == (r <= thr), (float(x), r, thr, eps)
    assert decided > 0.5 * len(xs) * 2 * 5
