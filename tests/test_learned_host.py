"""Host logic of the learned smoother parameters: target selection and parameter maps
(no GPU: pure Python on measured-rate dictionaries)."""
from paper_1603_02524_gb300 import learned


def rates_with_cliff(best=1.2, cliff=1.3):
    """Rates that fall towards omega = best and jump to 1 (breakdown) from omega = cliff."""
    r = {}
    for om in learned.OMEGAS:
        for ta in learned.TAUS:
            base = 0.05 + 0.1 * abs(om - best) + (0.001 if ta == 0.5 else 0.0)
            r[(om, ta)] = 1.0 if om >= cliff - 1e-9 else base
    return r


def test_robust_best_keeps_a_margin_from_the_cliff():
    r = rates_with_cliff(best=1.25, cliff=1.3)
    om, ta = learned.robust_best(r)
    # 1.25 has the cliff within 0.1: the choice backs off to an omega whose neighbourhood is safe
    assert om <= 1.2 + 1e-9 and ta == 1.0


def test_robust_best_never_exceeds_the_target_cap():
    r = {(om, ta): 0.5 - 0.1 * om for om in learned.OMEGAS for ta in learned.TAUS}   # keeps improving
    om, _ = learned.robust_best(r)
    assert om <= learned.OMEGA_TARGET_MAX + 1e-9


def test_robust_best_prefers_the_paper_parameters_when_flat():
    r = {(om, ta): 0.1 for om in learned.OMEGAS for ta in learned.TAUS}
    r[(1.0, 1.0)] = 0.0999
    assert learned.robust_best(r) == (1.0, 1.0)


def test_parameter_maps_round_trip():
    """omega = 0.5 + 1.5 sigmoid(y0), tau = 0.1 + 0.9 sigmoid(y1), inverted by to_raw (within
    its clip to (1e-3, 1 - 1e-3) of the sigmoid range)."""
    import numpy as np
    for om in (0.6, 1.0, 1.3, 1.9):
        for ta in (0.15, 0.5, 0.99):
            y = learned.to_raw(om, ta)
            o2, t2 = learned.to_params(np.array([y], dtype=np.float64))
            assert abs(o2[0] - om) < 1e-5 and abs(t2[0] - ta) < 1e-5
