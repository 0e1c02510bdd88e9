"""The oracle against a number the paper prints about the model's dynamics:
its landscape holds a pathological fixed point around 190 Hz, where the
neurons fire again as soon as their refractory period ends (Sec. "Pathology
and the effect of modulating the propagation speed of action potentials
through the connectome").

On the synthetic 68-region connectome, strong coupling (g = 0.9) drives all
but the two most weakly connected regions onto that fixed point for every
adaptation strength b_e in {0, 60, 120} pA: rates constant in time, between
185 and 200 Hz, and below the 200 Hz clamp of E, so the value comes from the
transfer function's saturation (a transfer function off by a factor 2, for
instance, lands on the clamp or near 100 Hz)."""
import numpy as np

from paper_2311_13337_gb300 import synth


def test_pathological_fixed_point_near_190_hz(oracle):
    W, L = synth.connectome(68)
    prm = oracle.expand_grid([("g", [0.9]), ("b_e", [0.0, 60.0, 120.0]), ("w_noise", [1e-6])])
    m = oracle.make_model()
    r = oracle.simulate(m, W, L, prm, 0.1, 30000, 10, 1, want_state=False)
    E = r["E"][..., 2000:] * 1e3                      # Hz, the last second
    rate = E.mean(axis=2)
    active = rate > 50.0
    assert active.mean(axis=1).min() >= 0.95
    assert 185.0 <= np.median(rate[active]) < 200.0
    assert rate[active].max() < 0.999 * m.E_max * 1e3  # below the clamp
    assert E.std(axis=2)[active].max() < 0.5           # a fixed point, not an oscillation
