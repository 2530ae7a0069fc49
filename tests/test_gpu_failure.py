"""Failure detection on the host side of the C ABI, with no GPU fault: argument errors, non-finite
inputs found by a device-side check, injected allocation failures inside an HHS step (the step is
transactional and restores the state), and the interaction-list regrowth path forced by tiny
capacity estimates.  Every failure is made on the host (tg_debug_control) or by the caller's data."""
import numpy as np
import pytest
import torch

from paper_1712_10116_gb300 import ics

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1712_10116_gb300 import binding as tg
    DEV = torch.device("cuda:0")


def _sentinel(shape):
    return torch.full(shape, 12345.0, dtype=torch.float64, device=DEV)


def test_argument_errors_leave_outputs_untouched():
    pos, _, mass = ics.plummer(500, 1001)
    P = torch.tensor(pos, device=DEV)
    M = torch.tensor(mass, device=DEV)
    s = tg.Solver(tg.Params(p=4, n_crit=32))
    acc, pot = _sentinel((3, 500)), _sentinel((500,))
    rc = tg.load().tg_fmm_forces(s.ctx, -1, tg._ptr(P), tg._ptr(M), None, tg._ptr(acc), tg._ptr(pot))
    assert rc == -1
    host = np.zeros(3 * 500)   # host memory where device memory is required
    rc = tg.load().tg_fmm_forces(s.ctx, 500, host.ctypes.data, tg._ptr(M), None, tg._ptr(acc), tg._ptr(pot))
    assert rc == -1
    rc = tg.load().tg_fmm_forces(s.ctx, 500, tg._ptr(P), None, None, tg._ptr(acc), tg._ptr(pot))
    assert rc == -1
    torch.cuda.synchronize()
    assert bool((acc == 12345.0).all()) and bool((pot == 12345.0).all())
    with pytest.raises(tg.TGError):
        tg.tg_hhs_step(s.ctx)   # before tg_hhs_init: TG_ERR_STATE
    with pytest.raises(tg.TGError):
        tg.tg_debug_control(s.ctx, 99, 0)
    s.close()


@pytest.mark.parametrize("what", ["nan_pos", "inf_pos", "nan_mass"])
def test_nonfinite_inputs_are_rejected(what):
    pos, vel, mass = ics.plummer(2000, 1001)
    if what == "nan_pos":
        pos[1, 777] = np.nan
    elif what == "inf_pos":
        pos[2, 5] = -np.inf
    else:
        mass[1999] = np.nan
    P, V, M = (torch.tensor(a, device=DEV) for a in (pos, vel, mass))
    s = tg.Solver(tg.Params(p=4, n_crit=32))
    acc, pot = _sentinel((3, 2000)), _sentinel((2000,))
    with pytest.raises(tg.TGError, match="NONFINITE"):
        tg.tg_fmm_forces(s.ctx, P, M, None, acc, pot)
    torch.cuda.synchronize()
    assert bool((acc == 12345.0).all()) and bool((pot == 12345.0).all())
    with pytest.raises(tg.TGError, match="NONFINITE"):
        s.hhs_init(P, V, M)
    s.close()


def test_hhs_step_refuses_a_nonfinite_state_and_changes_nothing():
    pos, vel, mass = ics.plummer(2000, 1001)
    P, V, M = (torch.tensor(a, device=DEV) for a in (pos, vel, mass))
    s = tg.Solver(tg.Params(p=4, n_crit=32, dt_max=1 / 64, k_max=6))
    s.hhs_init(P, V, M)
    s.hhs_step()
    P[0, 11] = float("nan")
    P_before, V_before = P.clone(), V.clone()
    state_before = tg.tg_hhs_state(s.ctx, 2000, DEV, with_total=True)
    with pytest.raises(tg.TGError, match="NONFINITE"):
        s.hhs_step()
    torch.cuda.synchronize()
    assert torch.equal(P.isnan(), P_before.isnan())
    assert torch.equal(torch.nan_to_num(P), torch.nan_to_num(P_before)) and torch.equal(V, V_before)
    for a, b in zip(tg.tg_hhs_state(s.ctx, 2000, DEV, with_total=True), state_before):
        assert torch.equal(a, b)
    s.close()


def _plummer_state(n=3000):
    pos, vel, mass = ics.plummer(n, 1001)
    return (torch.tensor(a, device=DEV) for a in (pos, vel, mass))


def test_injected_allocation_failure_inside_a_step_is_transactional():
    prm = tg.Params(p=4, n_crit=32, dt_max=1 / 16, k_max=6, kernel=tg.TG_KERNEL_PLUMMER)
    # reference: one step without injection
    P0, V0, M = _plummer_state()
    ref = tg.Solver(prm)
    Pr, Vr = P0.clone(), V0.clone()
    ref.hhs_init(Pr, Vr, M)
    ref.hhs_step()
    torch.cuda.synchronize()
    failures = 0
    for allowed in range(0, 64):
        s = tg.Solver(prm)
        P, V = P0.clone(), V0.clone()
        s.hhs_init(P, V, M)
        state0 = tg.tg_hhs_state(s.ctx, P.shape[1], DEV, with_total=True)
        tg.tg_debug_control(s.ctx, tg.TG_DEBUG_FAIL_ALLOC, allowed)
        try:
            s.hhs_step()
        except tg.TGError as e:
            assert "OOM" in str(e)
            failures += 1
            torch.cuda.synchronize()
            # nothing changed: positions, velocities, integrator state
            assert torch.equal(P, P0) and torch.equal(V, V0)
            for a, b in zip(tg.tg_hhs_state(s.ctx, P.shape[1], DEV, with_total=True), state0):
                assert torch.equal(a, b)
            # with the injection off the same context completes the step like the reference
            tg.tg_debug_control(s.ctx, tg.TG_DEBUG_FAIL_ALLOC, -1)
            s.hhs_step()
            torch.cuda.synchronize()
            assert torch.allclose(P, Pr, rtol=0, atol=1e-13) and torch.allclose(V, Vr, rtol=0, atol=1e-12)
            s.close()
            continue
        s.close()
        break
    assert failures >= 1, "the first step of a fresh context allocates: some injection must fail it"


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_interaction_lists_regrow_from_tiny_capacities(precision):
    pos, _, mass = ics.clustered(20000, 1007)
    P = torch.tensor(np.ascontiguousarray(pos), device=DEV)
    M = torch.tensor(mass, device=DEV)
    prec = tg.TG_PREC_FP64 if precision == "fp64" else tg.TG_PREC_FP32
    prm = tg.Params(p=4, n_crit=32, precision=prec)
    a_ref, _ = tg.Solver(prm).fmm_forces(P, M)
    s = tg.Solver(prm)
    tg.tg_debug_control(s.ctx, tg.TG_DEBUG_LIST_CAPACITY, 1)   # 0.001 list entries per cell
    a, _ = s.fmm_forces(P, M)
    assert s.stats()["list_regrowths"] >= 1
    # float32: two runs of the same evaluation differ in the order of their float atomics, each within the
    # float32 parity bound of the exact result: compare against max(|a|, 0.1 median |a|) like the parity tests
    nb = torch.linalg.norm(a_ref, dim=0)
    scale = nb if precision == "fp64" else torch.maximum(nb, 0.1 * nb.median())
    rel = (torch.linalg.norm(a - a_ref, dim=0) / scale).max().item()
    assert rel < (1e-13 if precision == "fp64" else 1e-5), rel
    s.close()
