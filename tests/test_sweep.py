"""Step-count / stability / grid-saving studies (paper_2208_03562_gb300.sweep).

CPU tests check the experiment table against the paper's printed grids and
the definitions of Ma, Re and the lid speed. The GPU test checks the two
claims of Sec. 5.2 that need no external data: preconditioning (gamma < 1)
cuts the steps to a residual by a large factor, and it leaves the steady
field unchanged.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2208_03562_gb300 import sweep as SW

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_experiments_match_the_printed_grids():
    with open(os.path.join(GOLDEN, "paper_grids.json")) as fh:
        cases = json.load(fh)["cases"]
    printed = {(c["nx"], c["ny"], c["r"]) for c in cases}
    for e in SW.PAPER_EXPERIMENTS:
        assert (e.nx, e.ny, round(e.r, 2)) in printed, e.name
        # Sec. 5.2: r = AR Nx / Ny
        assert abs(e.ar * e.nx / e.ny - e.r) < 1e-2


def test_lid_speed_and_viscosity_from_mach_and_reynolds():
    e = SW.PAPER_EXPERIMENTS[0]  # shallow, r = 0.2, Ma = 0.06, Re = 100
    assert math.isclose(e.u_lid, 0.06 * 0.2 / math.sqrt(3.0), rel_tol=1e-15)  # Ma = U / (q c_s*), q = r < 1
    assert math.isclose(e.u_lid * e.ny * e.r / e.nu, e.re, rel_tol=1e-12)      # Re = U H / nu, H = ny r
    d = SW.PAPER_EXPERIMENTS[2]  # deep, r = 1.6 > 1: q = 1
    assert math.isclose(d.u_lid, 0.06 / math.sqrt(3.0), rel_tol=1e-15)


def test_centreline_profiles_pick_the_middle():
    ny, nx = 6, 5
    ux = np.tile(np.arange(nx, dtype=float), (ny, 1))
    uy = np.tile(np.arange(ny, dtype=float)[:, None], (1, nx))
    ys, u_c, xs, v_c = SW.centreline_profiles((None, ux, uy), nx, ny, 1.0)
    assert np.all(u_c == 2.0)               # odd nx: the middle column
    assert np.all(v_c == 2.5)               # even ny: mean of the two middle rows
    assert np.allclose(ys, (np.arange(ny) + 0.5) / ny)


@pytest.mark.gpu
def test_preconditioning_cuts_steps_and_keeps_the_steady_field():
    """Shallow cavity of Sec. 5.2 (r = 0.2, 100 x 125, Re = 100, Ma = 0.06)
    to residual 1e-6. The smaller gamma, the fewer steps (about x3 at
    gamma = 0.1 at this residual; the reduction grows as the residual target
    tightens). The steady field is the same for every gamma up to O(Ma^2 /
    gamma)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    e = SW.Experiment("shallow_Ma0.06", "Sec. 5.2", 0.25, 0.2, 100, 125, 100.0, 0.06, (1.0, 0.5, 0.1))
    res = SW.convergence_study(e, tol=1e-6, want_fields=True, max_steps=4_000_000)
    runs = res["runs"]
    assert all(r["status"] == "converged" for r in runs)
    steps = [r["steps"] for r in runs]
    assert steps[0] > steps[1] > steps[2], steps
    assert runs[2]["step_reduction_vs_gamma1"] > 2.5, steps
    # the steady states of the preconditioned equations coincide up to the
    # weak-compressibility error: p = gamma c_s^2 rho makes density
    # variations 1/gamma larger, an O(Ma^2 / gamma) effect (0.0036 / gamma)
    _, u1, v1 = runs[0]["fields"]
    for r in runs[1:]:
        _, u2, v2 = r["fields"]
        rel = math.sqrt(np.sum((u1 - u2) ** 2 + (v1 - v2) ** 2) / np.sum(u1 ** 2 + v1 ** 2))
        assert rel < 0.006 / r["gamma"], (r["gamma"], rel)


@pytest.mark.gpu
def test_rectangular_grid_reproduces_the_square_grid():
    """Sec. 5.2: the shallow cavity (AR = 0.25, Re 100, Ma 0.06) on 100 x 125
    nodes with r = 0.2 and on 400 x 100 nodes with r = 1 reaches the same
    steady state: the centre-line velocity profiles agree to within 1 % of
    the lid speed (the two grids have different spacings, so they agree to
    their discretisation error, not to round-off)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    res = SW.grid_saving_study(tol=1e-7)
    assert all(r["status"] == "converged" for r in res["runs"].values())
    assert res["max_abs_diff_u_centreline_over_U"] < 0.01
    assert res["max_abs_diff_v_centreline_over_U"] < 0.01
    assert res["nodes"]["rect_r0.2_100x125"] * 3 < res["nodes"]["square_r1_400x100"]


@pytest.mark.gpu
def test_central_moments_stay_stable_where_raw_moments_diverge():
    """Sec. 5.3: on the 100 x 100, r = 0.25 cavity at gamma = 0.2 and
    U = 0.02, Re = 1800 lies between the stability limits of the two schemes
    (raw moments about 1.6e3, central moments about 2.0e3): the central-moment
    run stays finite for 200,000 steps, the raw-moment run diverges."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    nx = ny = 100
    r, gamma, u, re = 0.25, 0.2, 0.02, 1800.0
    nu = u * ny * r / re
    prc = SW.solve(nx, ny, r, gamma, nu, u, 1e-9, 200_000, "f32", model=0)
    prnr = SW.solve(nx, ny, r, gamma, nu, u, 1e-9, 200_000, "f32", model=1)
    assert prc["status"] != "diverged", prc
    assert prnr["status"] == "diverged", prnr


def _study_oracle():
    with open(os.path.join(GOLDEN, "study_oracle.json")) as fh:
        return json.load(fh)["runs"]


def _proj_rel(rec, fields):
    """Relative L2 distance of (u_x, u_y) from the oracle's, estimated from the
    stored random projections (their mean square difference estimates the
    squared distance)."""
    from paper_2208_03562_gb300 import inputs as I
    _, ux, uy = fields
    w = I.projection_signs(rec["proj_seed"], len(rec["proj"]), rec["nx"], rec["ny"])
    p = np.array([np.sum(w[k, 0] * ux) + np.sum(w[k, 1] * uy) for k in range(len(rec["proj"]))])
    return math.sqrt(np.mean((p - np.array(rec["proj"])) ** 2)) / math.hypot(rec["norm_ux"], rec["norm_uy"])


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["shallow_gamma1", "shallow_gamma0.1"])
def test_convergence_study_on_the_fp64_path_reproduces_the_oracle(name):
    """The convergence study's solve (sweep.solve) on the FP64 path against
    the FP64 oracle's run of the same shallow cavity (Sec. 5.2: 100 x 125,
    r = 0.2, Re 100, Ma 0.06) to the residual 1e-8: the same step count to
    the step, and the same steady field to the FP64 parity bar (1e-10)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    rec = _study_oracle()[name]
    r = SW.solve(rec["nx"], rec["ny"], rec["r"], rec["gamma"], rec["nu"], rec["u_lid"], rec["tol"], 5_000_000,
                 "f64", want_fields=True)
    assert r["status"] == "converged" and rec["status"] == "converged"
    assert r["steps"] == rec["steps"], (r["steps"], rec["steps"])
    assert abs(r["residual"] - rec["residual"]) <= 1e-6 * rec["residual"]
    assert _proj_rel(rec, r["fields"]) <= 1e-10


@pytest.mark.gpu
def test_grid_saving_study_on_the_fp64_path_reproduces_the_oracle():
    """The grid-saving study (sweep.grid_saving_study) on the FP64 path: both
    grids take the oracle's step counts to the residual 1e-7, and the
    centre-line differences the study reports equal those of the oracle's
    profiles to 1e-10 of the lid speed."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    recs = _study_oracle()
    res = SW.grid_saving_study(tol=1e-7, dtype="f64")
    prof = {}
    for name in ("rect_r0.2_100x125", "square_r1_400x100"):
        run, rec = res["runs"][name], recs[name]
        assert run["status"] == "converged" and run["steps"] == rec["steps"], (name, run["steps"], rec["steps"])
        prof[name] = rec
    a, b = prof["rect_r0.2_100x125"], prof["square_r1_400x100"]
    ys_a = (np.arange(a["ny"]) + 0.5) / a["ny"]
    ys_b = (np.arange(b["ny"]) + 0.5) / b["ny"]
    xs_a = (np.arange(a["nx"]) + 0.5) / a["nx"]
    xs_b = (np.arange(b["nx"]) + 0.5) / b["nx"]
    du = np.max(np.abs(np.array(a["u_centre"]) / a["u_lid"] -
                       np.interp(ys_a, ys_b, np.array(b["u_centre"]) / b["u_lid"])))
    dv = np.max(np.abs(np.array(a["v_centre"]) / a["u_lid"] -
                       np.interp(xs_a, xs_b, np.array(b["v_centre"]) / b["u_lid"])))
    assert abs(res["max_abs_diff_u_centreline_over_U"] - du) <= 1e-10
    assert abs(res["max_abs_diff_v_centreline_over_U"] - dv) <= 1e-10
