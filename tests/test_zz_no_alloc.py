"""The allocation-free entry point (mppi_solve_noalloc), for callers that
cannot allocate device memory (a real-time loop that forbids allocation
after start-up, a plug-in whose host framework owns all device memory).

It is checked through the C ABI against the handle-based entry point
(mppi_solve_async) on the same inputs, within the parity tolerance, on two
calls in a row of different sizes (the second call reuses the fixed scratch
array the first one left behind).  This file is collected last so that a
run stopping at the first failure has already run every other test."""
import os

import numpy as np
import pytest

from parity import COST_RTOL, U_RTOL, control_err, cost_err, state_err

pytestmark = pytest.mark.gpu


def _run(mppi, torch, prob, noalloc: bool):
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    K, N = prob["params"]["K"], prob["params"]["N"]
    ins = (t(prob["x_hat"]), t(prob["ref"]), t(prob["obstacles"]) if prob["obstacles"].size else None,
           t(prob["u_nom"]))
    out = {k: torch.zeros(n, dtype=torch.float32, device=dev) for k, n in
           (("u_out", (N, 4)), ("u_cmd", 4), ("u_next", (N, 4)), ("x_next", 13), ("costs", K))}
    status = torch.full((1,), -99, dtype=torch.int32, device=dev)
    if noalloc:
        mppi.solve_noalloc(prob["model"], prob["params"], *ins, prob["iter"], status=status, **out)
    else:
        s = mppi.Solver(prob["model"], prob["params"])
        s.solve_async(*ins, prob["iter"], status=status, **out)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["status"] = int(status.item())
    if not noalloc:
        s.close()
    return res


def test_noalloc_matches_handle_entry_point_twice():
    import torch
    assert torch.cuda.is_available()
    from paper_2407_09812_gb300 import build as B
    B.build()
    from paper_2407_09812_gb300 import inputs as I
    from paper_2407_09812_gb300 import mppi

    first = I.eight_with_spheres(K=4096, N=60, M=48, t0=0.8, **{"lambda": 200.0})
    second = I.eight_with_spheres(K=777, N=13, M=9, t0=2.1, seed=3)
    second["iter"] = 5
    for prob in (first, second):
        ref = _run(mppi, torch, prob, noalloc=False)
        got = _run(mppi, torch, prob, noalloc=True)
        assert got["status"] == 0 and ref["status"] == 0
        sig = prob["params"]["sigma"]
        assert control_err(got["u_out"], ref["u_out"], sig) <= U_RTOL
        assert control_err(got["u_next"], ref["u_next"], sig) <= U_RTOL
        assert control_err(got["u_cmd"], ref["u_cmd"], sig) <= U_RTOL
        assert state_err(got["x_next"], ref["x_next"]) <= U_RTOL
        assert cost_err(got["costs"], ref["costs"])[0] <= COST_RTOL


def test_noalloc_at_its_scratch_limits_matches_the_oracle():
    """K = 32768 and N = 256 fill the fixed scratch exactly (256 tiles of
    128 samples, 4 + 4N floats each, after the 256-byte header).  The
    result at those sizes is compared with the handle-based entry point and
    with the FP64 oracle directly, within the parity tolerance."""
    import torch
    from oracle import oracle as O
    from paper_2407_09812_gb300 import inputs as I
    from paper_2407_09812_gb300 import mppi
    prob = I.eight_with_spheres(K=32768, N=256, dt=0.004, M=12, t0=1.1, **{"lambda": 300.0})
    got = _run(mppi, torch, prob, noalloc=True)
    ref = _run(mppi, torch, prob, noalloc=False)
    orc = O.mppi_step(prob, n_threads=os.cpu_count() or 1)
    assert got["status"] == 0 and ref["status"] == 0
    sig = prob["params"]["sigma"]
    for want in (ref, orc):
        assert control_err(got["u_out"], want["u_out"], sig) <= U_RTOL
        assert control_err(got["u_next"], want["u_next"], sig) <= U_RTOL
        assert control_err(got["u_cmd"], want["u_cmd"], sig) <= U_RTOL
        assert cost_err(got["costs"], want["costs"], want.get("min_gap"))[0] <= COST_RTOL
    assert state_err(got["x_next"], ref["x_next"]) <= U_RTOL


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2407_09812_gb300 import inputs as I
    from paper_2407_09812_gb300 import mppi
    x = torch.zeros(13, device="cuda")
    big = I.plain_hover(K=32769, N=10)
    with pytest.raises(mppi.MppiError) as e:
        mppi.solve_noalloc(big["model"], big["params"], x, torch.zeros(11, 13, device="cuda"), None,
                           torch.zeros(10, 4, device="cuda"), 0)
    assert e.value.code == mppi.EINVAL
    long = I.plain_hover(K=100, N=257)
    with pytest.raises(mppi.MppiError) as e:
        mppi.solve_noalloc(long["model"], long["params"], x, torch.zeros(258, 13, device="cuda"), None,
                           torch.zeros(257, 4, device="cuda"), 0)
    assert e.value.code == mppi.EINVAL
    # Buffers that do not match K and N are refused before any call.
    ok = I.plain_hover(K=100, N=10)
    with pytest.raises(ValueError):
        mppi.solve_noalloc(ok["model"], ok["params"], x, x, None, x, 0)
