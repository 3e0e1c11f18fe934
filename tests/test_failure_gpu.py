"""Failure path on the GPU without a GPU fault: the kernel's bounded
device-side waits run out (the obstacle staging copy is skipped, so its
mbarrier never completes), the step reports MPPI_ETIMEOUT to the host, and
the same handle and context then solve correctly again."""
import numpy as np
import pytest

from parity import assert_step_close

pytestmark = pytest.mark.gpu

POLLS = 256  # a short bound: each timed-out wait ends within microseconds


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available()
    from paper_2407_09812_gb300 import build as B
    B.build()
    from paper_2407_09812_gb300 import mppi
    return mppi


@pytest.mark.parametrize("shape", [(128, 1, 0), (128, 2, 0), (256, 1, 1), (384, 1, 2), (512, 1, 3),
                                   (128, 1, 0, 0.0, 2)])
def test_timeout_reported_and_context_stays_usable(M, orc, inp, shape):
    prob = inp.eight_with_spheres(K=3000, N=24, M=32, t0=0.3, **{"lambda": 50.0})
    s = M.Solver(prob["model"], prob["params"])
    s.set_shape(*shape)
    args = (prob["x_hat"], prob["ref"], prob["obstacles"], prob["u_nom"], prob["iter"])
    s.set_wait_limit(POLLS, stall_obstacle_copy=True)
    for _ in range(2):  # the per-instance counters are left clean for the next launch
        with pytest.raises(M.MppiError) as e:
            s.solve(*args)
        assert e.value.code == M.ETIMEOUT
    s.set_wait_limit(0, stall_obstacle_copy=False)
    out = s.solve(*args, want_costs=True)
    assert out["status"] == M.OK
    assert_step_close(prob, out, orc.mppi_step(prob, n_threads=8))
    s.close()


def test_timeout_in_a_batched_graph_flags_instances_then_recovers(M, orc, inp):
    import torch
    probs = inp.batched_uneven(n=8, seed=3, K_range=(200, 2500), N_range=(4, 30), M_max=24, **{"lambda": 50.0})
    for i, p in enumerate(probs):
        if i % 2 == 0:
            p["obstacles"] = np.zeros((0, 4), np.float32)
    cap = {"max_instances": len(probs), "max_samples": sum(p["params"]["K"] for p in probs),
           "N_max": max(p["params"]["N"] for p in probs), "M_max": 64}
    s = M.Solver(probs[0]["model"], probs[0]["params"], cap)
    dev = torch.device("cuda")

    def insts():
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        out = []
        for p in probs:
            K, N = p["params"]["K"], p["params"]["N"]
            out.append({"x_hat": t(p["x_hat"]), "ref": t(p["ref"]), "u_nom": t(p["u_nom"]),
                        "obstacles": t(p["obstacles"]) if p["obstacles"].size else None,
                        "u_out": torch.zeros(N, 4, device=dev), "u_cmd": torch.zeros(4, device=dev),
                        "u_next": torch.zeros(N, 4, device=dev), "x_next": torch.zeros(13, device=dev),
                        "status": torch.full((1,), 99, dtype=torch.int32, device=dev),
                        "K": K, "N": N, "dt": p["params"]["dt"], "lambda": p["params"]["lambda"],
                        "sigma": p["params"]["sigma"], "seed": p["params"]["seed"],
                        "stream_id": p["params"]["stream_id"], "iter": p["iter"]})
        return out

    s.set_wait_limit(POLLS, stall_obstacle_copy=True)
    ins = insts()
    s.solve_batch(ins, graph=True)
    torch.cuda.synchronize()
    for p, d in zip(probs, ins):
        st = int(d["status"].item())
        if p["obstacles"].size:
            assert st == M.ETIMEOUT
        else:  # untouched by a timed-out block: a correct step; else flagged
            assert st in (M.OK, M.ETIMEOUT)
            if st == M.OK:
                got = {k: d[k].cpu().numpy() for k in ("u_out", "u_cmd", "u_next", "x_next")}
                assert_step_close(p, got, orc.mppi_step(p, n_threads=8))
    s.set_wait_limit(0, stall_obstacle_copy=False)
    ins = insts()
    s.solve_batch(ins, graph=True)
    torch.cuda.synchronize()
    for p, d in zip(probs, ins):
        assert int(d["status"].item()) == M.OK
        got = {k: d[k].cpu().numpy() for k in ("u_out", "u_cmd", "u_next", "x_next")}
        assert_step_close(p, got, orc.mppi_step(p, n_threads=8))
    s.close()
