"""The sampling step (Sec. III-A: delta u_{k,j} ~ N(0, Sigma)) on the GPU,
through the C ABI (mppi_sample_noise), against the oracle's FP64 noise
element by element, and against the noise a solve actually applies.

Tolerance, from the arithmetic of the GPU form.  With z = delta / sigma and
r the Box-Muller radius of z's pair (r^2 = z_0^2 + z_1^2, resp. z_2^2 +
z_3^2, taken from the oracle): the radius sqrt(-2 ln u) carries a relative
error below 1.3e-6 (hardware log2 away from u = 1, a four-term series near
it, the square root as x rsqrt(x)), the hardware sine and cosine of an
angle in (-pi, pi) an absolute error below 2^-21.4 (3.6e-7), the product
one rounding; so |z_gpu - z| <= r (1.3e-6 + 3.6e-7 + 6e-8) < 2e-6 r, and
delta = sigma z adds one more rounding (6e-8 relative).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2407_09812_gb300 import build as B
    B.build()
    from paper_2407_09812_gb300 import mppi
    mppi.lib()
    return mppi


def noise_bound(ref, sigma):
    """Per-element bound on |delta_gpu - delta| (module docstring)."""
    z = ref / sigma
    r01 = np.hypot(z[..., 0], z[..., 1])
    r23 = np.hypot(z[..., 2], z[..., 3])
    r = np.stack([r01, r01, r23, r23], axis=-1)
    return sigma * 2e-6 * r + 6e-8 * np.abs(ref) + 1e-12


def check_noise(got, ref, sigma):
    err = np.abs(got.astype(np.float64) - ref)
    bound = noise_bound(ref, sigma)
    worst = float(np.max(err / bound))
    assert worst <= 1.0, (worst, np.unravel_index(np.argmax(err / bound), err.shape))
    return worst


@pytest.mark.parametrize("K,N,it", [(16384, 100, 7), (1000, 37, (1 << 33) + 5), (1, 1, 0), (257, 1024, 3)])
def test_noise_matches_oracle_element_by_element(M, orc, inp, K, N, it):
    """Every element of delta for samples 0..K-1 against the oracle's
    independent Philox4x32-10 and FP64 Box-Muller; (16384, 100) is the
    closed-loop workload in full, (257, 1024) the longest horizon, and the
    iteration count crosses the counter's 32-bit word."""
    p = inp.params(K=K, N=N, seed=0x1234_5678_9ABC, stream_id=11)
    sigma = np.asarray(p["sigma"], dtype=np.float64)
    got = M.sample_noise(p, it, 0, K, N).cpu().numpy()
    ref = orc.noise_block(p, it, K, N)
    check_noise(got, ref, sigma)
    # The draws really are standard normal at this size (loose moments).
    if K * N >= 1 << 20:
        z = got / sigma.astype(np.float32)
        assert abs(float(z.mean())) < 5e-3 and abs(float(z.var()) - 1.0) < 5e-3


@pytest.mark.parametrize("k0,K,N", [(1 << 24, 4096, 2), ((1 << 32) - 300, 300, 3), (123_457, 200, 20)])
def test_noise_at_the_top_of_the_sample_range(M, orc, inp, k0, K, N):
    """Sample indices far from 0 (up to the last one of the 32-bit counter
    word): each element against the oracle's noise for that (k, j)."""
    p = inp.params(seed=99, stream_id=3)
    sigma = np.asarray(p["sigma"], dtype=np.float64)
    got = M.sample_noise(p, 17, k0, K, N).cpu().numpy()
    rng = np.random.default_rng(5)
    ks = np.unique(np.concatenate([[0, K - 1], rng.integers(0, K, 60)]))
    ref = np.stack([np.stack([orc.noise(p, 17, int(k0 + k), j) for j in range(N)]) for k in ks])
    check_noise(got[ks], ref, sigma)


def test_solve_applies_the_sampled_noise(M, inp):
    """With one rollout its weight is exactly 1, so the update of Eq.
    u_update is u_nom + delta_0 (to one rounding): the solve draws the same
    noise the entry point returns."""
    prob = inp.plain_hover(K=1, N=24)
    p = prob["params"]
    s = M.Solver(prob["model"], p)
    out = s.solve(prob["x_hat"], prob["ref"], prob["obstacles"], prob["u_nom"], prob["iter"])
    s.close()
    d = M.sample_noise(p, prob["iter"], 0, 1, p["N"]).cpu().numpy()[0]
    want = prob["u_nom"].astype(np.float32) + d
    assert np.all(np.abs(out["u_out"] - want) <= 2 * np.spacing(np.abs(want))), np.max(np.abs(out["u_out"] - want))


def test_noise_is_deterministic_and_stream_separated(M, inp):
    p = inp.params(seed=4, stream_id=0)
    a = M.sample_noise(p, 9, 0, 512, 16).cpu().numpy()
    b = M.sample_noise(p, 9, 0, 512, 16).cpu().numpy()
    assert np.array_equal(a, b)
    c = M.sample_noise(dict(p, stream_id=1), 9, 0, 512, 16).cpu().numpy()
    d = M.sample_noise(p, 10, 0, 512, 16).cpu().numpy()
    assert not np.any(a == c) or np.mean(a == c) < 1e-3
    assert np.mean(a == d) < 1e-3
