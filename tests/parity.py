"""Comparison helpers for CUDA-vs-oracle parity tests.

Tolerances (FP32 kernel against the FP64 oracle on identical FP32 inputs):
* per-sample cost S_k: relative 1e-4;
* control update u_out (and the warm start, the command): 1e-4 relative per
  control, measured against max(|u_oracle|, sigma_c) so that body-rate
  entries passing through zero are judged on the scale of their noise;
* samples with a state whose collision test is within 1e-4 of its boundary
  (the state's smallest squared gap over the obstacles within 1e-4 m^2 of
  0, or its position within 1e-4 m of an occupancy-changing voxel face) are
  left out of the cost comparison, because the once-per-state collision
  indicator is discontinuous there; the update comparison keeps them;
* the plant state x_next is the plant step of the applied command, which is
  formed from u_out_0 (R26): it is compared, 1e-4 relative per component
  (floor 1e-3), with the oracle's plant step of the GPU's own u_out_0, so
  the comparison measures the step itself and does not re-measure the
  update's allowed error through it.
"""
import numpy as np

COST_RTOL = 1e-4
U_RTOL = 1e-4
GRAZE = 1e-4


def cost_err(c_gpu, c_orc, min_gap=None):
    c_gpu = np.asarray(c_gpu, np.float64)
    c_orc = np.asarray(c_orc, np.float64)
    keep = np.isfinite(c_orc)
    if min_gap is not None:
        keep &= ~(np.abs(np.asarray(min_gap)) < GRAZE)
    rel = np.abs(c_gpu[keep] - c_orc[keep]) / np.maximum(np.abs(c_orc[keep]), 1e-30)
    return (float(rel.max()) if rel.size else 0.0), int((~keep).sum())


def control_err(u_gpu, u_orc, sigma):
    u_gpu = np.asarray(u_gpu, np.float64).reshape(-1, 4)
    u_orc = np.asarray(u_orc, np.float64).reshape(-1, 4)
    scale = np.maximum(np.abs(u_orc), np.asarray(sigma, np.float64)[None, :])
    diff = np.abs(u_gpu - u_orc)
    with np.errstate(invalid="ignore", divide="ignore"):
        rel = np.where(diff == 0.0, 0.0, diff / np.maximum(scale, 1e-30))
    return float(rel.max())


def state_err(x_gpu, x_orc):
    x_gpu = np.asarray(x_gpu, np.float64)
    x_orc = np.asarray(x_orc, np.float64)
    return float((np.abs(x_gpu - x_orc) / np.maximum(np.abs(x_orc), 1e-3)).max())


def plant_step_of(prob, u0):
    """The oracle's x_next for the applied command formed from u0: clamp,
    constraint pipeline from x_hat, one RK4 step of shift_alpha * dt."""
    from oracle import oracle as O
    m, p = prob["model"], prob["params"]
    F, tau, _ = O.feasible_input(m, prob["x_hat"], O.clamp_input(m, np.asarray(u0, np.float64)), p["dt"])
    return O.rk4_step(m, prob["x_hat"], F, tau, p.get("shift_alpha", 1.0) * p["dt"])


def compare_step(prob, gpu: dict, orc: dict, check_costs=True):
    """Returns a dict of the worst relative errors of one step."""
    sigma = prob["params"]["sigma"]
    u_out = np.asarray(gpu["u_out"], np.float64).reshape(-1, 4)
    out = {
        "u_out": control_err(gpu["u_out"], orc["u_out"], sigma),
        "u_next": control_err(gpu["u_next"], orc["u_next"], sigma),
        "u_cmd": control_err(gpu["u_cmd"], orc["u_cmd"], sigma),
        "x_next": state_err(gpu["x_next"], plant_step_of(prob, u_out[0])),
        # Reported, not asserted: the plant step of the GPU's command against
        # the oracle's plant step of its own command (carries the update's
        # allowed error through one step of the model).
        "x_next_vs_oracle": state_err(gpu["x_next"], orc["x_next"]),
    }
    if check_costs and gpu.get("costs") is not None:
        out["costs"], out["grazing"] = cost_err(gpu["costs"], orc["costs"], orc.get("min_gap"))
    return out


# Worst errors seen by assert_step_close in this session (printed at the end
# of a GPU run by conftest).
WORST = {}


def assert_step_close(prob, gpu, orc, check_costs=True):
    e = compare_step(prob, gpu, orc, check_costs)
    for k, v in e.items():
        if k != "grazing":
            WORST[k] = max(WORST.get(k, 0.0), float(v))
    assert e["u_out"] <= U_RTOL, e
    assert e["u_next"] <= U_RTOL, e
    assert e["u_cmd"] <= U_RTOL, e
    assert e["x_next"] <= U_RTOL, e
    if "costs" in e:
        assert e["costs"] <= COST_RTOL, e
    return e
