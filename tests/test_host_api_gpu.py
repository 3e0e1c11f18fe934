"""The host-buffer solve (mppi_solve) replays [copy in, kernel, copy out]
from a CUDA graph from the second call of the same sizes on: replayed calls
give bitwise the results of uncaptured ones, a change of sizes or shape
recaptures, and the Philox counter passed each call is honoured."""
import numpy as np
import pytest

from parity import assert_step_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available()
    from paper_2407_09812_gb300 import build as B
    B.build()
    from paper_2407_09812_gb300 import mppi
    return mppi


def _solve(s, prob, it, obstacles=None):
    obs = prob["obstacles"] if obstacles is None else obstacles
    return s.solve(prob["x_hat"], prob["ref"], obs, prob["u_nom"], it, want_costs=True)


def test_graph_replay_equals_uncaptured_calls(M, orc, inp):
    prob = inp.eight_with_spheres(K=3000, N=30, M=24, t0=0.4, **{"lambda": 60.0})
    s = M.Solver(prob["model"], prob["params"])
    first = _solve(s, prob, prob["iter"])      # uncaptured
    _solve(s, prob, prob["iter"] + 1)          # uncaptured, then captured
    for it in (prob["iter"], prob["iter"] + 7, prob["iter"]):  # replayed
        out = _solve(s, prob, it)
        if it == prob["iter"]:
            for k in ("u_out", "u_cmd", "u_next", "x_next", "costs"):
                assert np.array_equal(out[k], first[k]), k
        else:
            assert_step_close(dict(prob, iter=it), out, orc.mppi_step(dict(prob, iter=it), n_threads=8))
    s.close()


def test_changed_sizes_and_shape_recapture(M, orc, inp):
    prob = inp.eight_with_spheres(K=2000, N=20, M=16, t0=0.8, **{"lambda": 60.0})
    s = M.Solver(prob["model"], prob["params"])
    for _ in range(3):
        _solve(s, prob, prob["iter"])
    fewer = prob["obstacles"][:5]
    p2 = dict(prob, obstacles=fewer)
    for _ in range(3):  # new obstacle count: plain, capture, replay
        out = _solve(s, p2, prob["iter"])
    assert_step_close(p2, out, orc.mppi_step(p2, n_threads=8))
    s.set_shape(128, 2, 0)
    for _ in range(3):  # new shape
        out = _solve(s, prob, prob["iter"])
    assert_step_close(prob, out, orc.mppi_step(prob, n_threads=8))
    s.close()


def test_shape_validation(M):
    from paper_2407_09812_gb300 import inputs as I
    prob = I.plain_hover(K=512, N=10)
    s = M.Solver(prob["model"], prob["params"])
    for bad in ((128, 3, 0), (100, 1, 0), (128, 4, 1), (64, 2, 1), (1024, 1, 0), (128, 1, 0, -1.0),
                (128, 1, 0, float("nan")), (256, 1, 0, 0.0, 2), (128, 2, 0, 0.0, 2), (128, 1, 1, 0.0, 2),
                (128, 1, 0, 0.0, 3)):
        with pytest.raises(M.MppiError):
            s.set_shape(*bad)
    s.set_shape(256, 32, 0, 0.5)
    assert s.get_shape(512, 10, 0) == (256, 32, 0, 0.5, 1)
    s.set_shape(64, 1, 0, 0.5, 2)
    assert s.get_shape(512, 10, 0) == (64, 1, 0, 0.5, 2)
    s.set_shape(0, 0, 0)
    assert s.get_shape(512, 10, 0)[:3] != (256, 32, 0)
    s.close()


def test_default_shapes(M):
    """Untuned sizes take the default for their tile count on this GPU's S
    SMs: at most one tile per SM, the split pipelined form with the smallest
    tile (32, 64, 128 samples) that keeps it so, unless its shared memory
    does not fit; at most two 128-sample tiles per SM with 16 or more
    obstacles, the two-warp pipelined form; from one 256-sample tile per SM
    on, two samples per thread unless the last wave of 256-sample tiles
    loads the SMs more than 8 % less evenly than 128-sample tiles; else one
    thread per sample."""
    import torch
    from paper_2407_09812_gb300 import inputs as I
    S = torch.cuda.get_device_properties(0).multi_processor_count
    prob = I.plain_hover(K=512, N=10)
    s = M.Solver(prob["model"], prob["params"])
    shape = lambda K, N, Mo: s.get_shape(K, N, Mo)[:3] + s.get_shape(K, N, Mo)[4:]
    assert shape(1024, 50, 0) == (128, 1, 3, 1)
    assert shape(32 * S, 100, 64) == (128, 1, 3, 1)
    assert shape(32 * S + 1, 100, 64) == (256, 1, 3, 1)
    assert shape(128 * S, 100, 0) == (512, 1, 3, 1)
    for K in (128 * S + 1, 256 * S):
        assert shape(K, 100, 64) == (256, 1, 1, 1), K
    assert shape(128 * S + 1, 100, 8) == (128, 1, 0, 1)
    assert shape(256 * S, 100, 8) == (128, 1, 0, 2)
    # 256 S + 1 samples: three 128-sample tiles on the busiest SM against two
    # 256-sample tiles (512 samples), one thread per sample; an exact
    # multiple of 256 S: two samples per thread.
    assert shape(256 * S + 1, 100, 64) == (128, 1, 0, 1)
    assert shape(7 * 256 * S, 200, 1024) == (128, 1, 0, 2)
    assert shape(1 << 22, 100, 32) == (128, 1, 0, 2)
    # The largest horizon with the largest obstacle set: the pipelined
    # forms' rings do not fit beside them, one thread per sample is taken.
    assert shape(1024, M.N_MAX, M.M_MAX) == (128, 1, 0, 1)
    s.close()


def test_plain_c_client_solves_like_the_binding(M, inp, tmp_path):
    """A C99 program that includes only include/mppi.h and links the library
    gets, through mppi_solve, bitwise the results of the Python binding."""
    import subprocess
    from c_client import build_client
    prob = inp.eight_with_spheres(K=2048, N=25, M=12, t0=0.6, **{"lambda": 40.0})
    exe = build_client(str(tmp_path))
    N, Mo = prob["params"]["N"], prob["obstacles"].shape[0]
    blob = (np.int32(Mo).tobytes() + bytes(M.make_model(prob["model"])) + bytes(M.make_params(prob["params"])) +
            np.ascontiguousarray(prob["x_hat"], np.float32).tobytes() +
            np.ascontiguousarray(prob["ref"], np.float32).tobytes() +
            np.ascontiguousarray(prob["obstacles"], np.float32).tobytes() +
            np.ascontiguousarray(prob["u_nom"], np.float32).tobytes() + np.uint64(prob["iter"]).tobytes())
    (tmp_path / "in.bin").write_bytes(blob)
    subprocess.run([exe, "solve", str(tmp_path / "in.bin"), str(tmp_path / "out.bin")], check=True)
    raw = (tmp_path / "out.bin").read_bytes()
    status = int(np.frombuffer(raw[:4], np.int32)[0])
    vals = np.frombuffer(raw[4:], np.float32)
    u_out, u_cmd = vals[:4 * N].reshape(N, 4), vals[4 * N:4 * N + 4]
    u_next, x_next = vals[4 * N + 4:8 * N + 4].reshape(N, 4), vals[8 * N + 4:8 * N + 17]
    s = M.Solver(prob["model"], prob["params"])
    ref = s.solve(prob["x_hat"], prob["ref"], prob["obstacles"], prob["u_nom"], prob["iter"])
    s.close()
    assert status == ref["status"] == 0
    for a, b in ((u_out, ref["u_out"]), (u_cmd, ref["u_cmd"]), (u_next, ref["u_next"]), (x_next, ref["x_next"])):
        assert np.array_equal(a, b)
