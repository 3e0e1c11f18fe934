"""Pins of the oracle's noise source (Sec. III-A: delta u ~ N(0, Sigma)).

* Philox4x32-10 bit patterns against an independent library implementation
  (Triton's Python-level Philox, run on the CPU by its interpreter).
* The uniform map is exact and stays in the open interval (0, 1).
* Box-Muller against its closed-form invariants and against scipy's normal
  distribution (Kolmogorov-Smirnov), plus moment and correlation checks.
"""
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest


_TRITON_SCRIPT = textwrap.dedent(
    """
    import os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def _k(out_ptr, c0p, c1p, c2p, c3p, seed, n, BLOCK: tl.constexpr):
        offs = tl.arange(0, BLOCK)
        m = offs < n
        c0 = tl.load(c0p + offs, mask=m)
        c1 = tl.load(c1p + offs, mask=m)
        c2 = tl.load(c2p + offs, mask=m)
        c3 = tl.load(c3p + offs, mask=m)
        r0, r1, r2, r3 = tl.random.philox(seed, c0, c1, c2, c3, 10)
        tl.store(out_ptr + offs * 4 + 0, r0, mask=m)
        tl.store(out_ptr + offs * 4 + 1, r1, mask=m)
        tl.store(out_ptr + offs * 4 + 2, r2, mask=m)
        tl.store(out_ptr + offs * 4 + 3, r3, mask=m)

    data = np.load(sys.argv[1])
    ctr, keys = data["ctr"], data["keys"]
    res = []
    for key, c in zip(keys, ctr):
        seed = int(key[1]) << 32 | int(key[0])
        cols = [torch.from_numpy(c[:, i].astype(np.uint32).view(np.int32).copy()) for i in range(4)]
        out = torch.zeros(4 * c.shape[0], dtype=torch.int32)
        _k[(1,)](out, *cols, seed, c.shape[0], BLOCK=c.shape[0])
        res.append(out.numpy().view(np.uint32).reshape(-1, 4))
    np.save(sys.argv[2], np.stack(res))
    """
)


def test_philox_matches_independent_library_implementation(orc, tmp_path):
    pytest.importorskip("triton")
    rng = np.random.default_rng(123)
    n_keys, n_ctr = 6, 64
    keys = rng.integers(0, 2**31, size=(n_keys, 2), dtype=np.uint64).astype(np.uint32)
    keys[0] = (0, 0)
    ctr = rng.integers(0, 2**32, size=(n_keys, n_ctr, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0, :4] = np.array([[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [0xFFFFFFFF] * 4], np.uint32)
    src = tmp_path / "in.npz"
    dst = tmp_path / "out.npy"
    np.savez(src, ctr=ctr, keys=keys)
    script = tmp_path / "tri.py"
    script.write_text(_TRITON_SCRIPT)
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, str(script), str(src), str(dst)], env=env, capture_output=True,
                       text=True, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
    ref = np.load(dst)
    for a in range(n_keys):
        for b in range(n_ctr):
            got = orc.philox(ctr[a, b], keys[a])
            assert np.array_equal(got, ref[a, b]), (a, b, got, ref[a, b])


def test_uniform_map_exact_open_interval(orc):
    for r in [0, 1, 511, 512, 0x7FFFFFFF, 0x80000000, 0xFFFFFE00, 0xFFFFFFFF]:
        u = orc.uniform(r)
        m = r >> 9
        assert u == (2 * m + 1) / 2.0**24
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u  # exactly representable in FP32


def test_box_muller_closed_form_invariants(orc):
    rng = np.random.default_rng(7)
    for u0, u1 in rng.uniform(1e-6, 1.0, size=(200, 2)):
        z0, z1 = orc.box_muller(u0, u1)
        assert math.isclose(z0 * z0 + z1 * z1, -2.0 * math.log(u0), rel_tol=1e-12, abs_tol=1e-14)
        ang = math.atan2(z1, z0) % (2 * math.pi)
        assert math.isclose(ang, (2 * math.pi * u1) % (2 * math.pi), rel_tol=0, abs_tol=1e-9)


@pytest.fixture(scope="module")
def normals(orc, inp):
    p = inp.params(K=512, N=256, sigma=(1.0, 1.0, 1.0, 1.0), seed=99, stream_id=3)
    d = orc.noise_block(p, 17, 512, 256)  # 512*256*4 = 524288 normals
    return d


def test_normals_distribution_ks_and_moments(normals):
    scipy_stats = pytest.importorskip("scipy.stats")
    z = normals.reshape(-1)
    n = z.size
    assert abs(z.mean()) < 6.0 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 6.0 * math.sqrt(2.0 / n)
    assert abs(scipy_stats.skew(z)) < 6.0 * math.sqrt(6.0 / n)
    assert abs(scipy_stats.kurtosis(z)) < 6.0 * math.sqrt(24.0 / n)
    assert scipy_stats.kstest(z, "norm").pvalue > 1e-4
    for c in range(4):
        assert scipy_stats.kstest(normals[..., c].reshape(-1), "norm").pvalue > 1e-4


def test_normals_uncorrelated_across_components_samples_and_steps(normals):
    bound = 6.0 / math.sqrt(normals[..., 0].size)

    def corr(a, b):
        a, b = a.reshape(-1), b.reshape(-1)
        return float(np.corrcoef(a, b)[0, 1])

    assert abs(corr(normals[..., 0], normals[..., 1])) < bound  # same Box-Muller pair
    assert abs(corr(normals[..., 0], normals[..., 2])) < bound
    assert abs(corr(normals[:-1, :, 0], normals[1:, :, 0])) < bound  # k vs k+1
    assert abs(corr(normals[:, :-1, 3], normals[:, 1:, 3])) < bound  # j vs j+1
    z2 = normals ** 2
    assert abs(corr(z2[..., 0], z2[..., 1])) < 2 * bound  # pair independence beyond linear


def test_uniform_words_chi_square(orc):
    scipy_stats = pytest.importorskip("scipy.stats")
    words = np.array([orc.philox((i, 5, 0, 0), (11, 22)) for i in range(40000)], dtype=np.uint64).reshape(-1)
    counts = np.bincount((words >> 24).astype(np.int64), minlength=256)
    assert scipy_stats.chisquare(counts).pvalue > 1e-4
    low = np.bincount((words & 0xFF).astype(np.int64), minlength=256)
    assert scipy_stats.chisquare(low).pvalue > 1e-4


def test_noise_scales_with_sigma_and_depends_on_every_counter_field(orc, inp):
    base = inp.params(sigma=(1.0, 1.0, 1.0, 1.0), seed=5, stream_id=2)
    d1 = orc.noise(base, 3, 10, 4)
    d2 = orc.noise(dict(base, sigma=(2.0, 0.5, 0.0, 4.0)), 3, 10, 4)
    assert np.allclose(d2, d1 * np.array([2.0, 0.5, 0.0, 4.0]), rtol=0, atol=0)
    assert np.all(orc.noise(dict(base, sigma=(0.0,) * 4), 3, 10, 4) == 0.0)
    variants = [orc.noise(base, 4, 10, 4), orc.noise(base, 3, 11, 4), orc.noise(base, 3, 10, 5),
                orc.noise(dict(base, seed=6), 3, 10, 4), orc.noise(dict(base, stream_id=3), 3, 10, 4),
                orc.noise(base, 3 + (1 << 32), 10, 4)]
    for v in variants:
        assert not np.allclose(v, d1)
