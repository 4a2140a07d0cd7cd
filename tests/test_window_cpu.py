"""The light-cone window construction used by the full-size GPU parity
test, checked on the oracle alone: a window run reproduces the periodic run
inside the cone that boundary effects cannot reach in the given steps."""
import numpy as np

from paper_2502_00920_gb300 import inputs as I


def run_oracle(O, case, steps, u0=None, v0=None):
    o = O.OracleSim(case, u0, v0)
    o.step(steps)
    return o.fields()


def test_light_cone_window_is_exact_on_the_oracle(oracle_mod):
    """The window construction itself: a window run of the oracle reproduces
    the full periodic oracle run inside the light cone (no GPU involved)."""
    case = I.roofline(n=96, nsteps=5)
    v0 = I.grf_velocity(case)
    full = run_oracle(oracle_mod, case, 5, None, v0)[0]
    margin, w, x0, y0 = 3 * 5 + 8, 16, 70, 40
    xs = np.arange(x0 - margin, x0 + w + margin) % 96
    ys = np.arange(y0 - margin, y0 + w + margin) % 96
    W = w + 2 * margin
    wcase = case.replace(nx=W, ny=W, dx=case.spacing, edges=(I.FREE,) * 4)
    win = run_oracle(oracle_mod, wcase, 5, None, v0[np.ix_(ys, xs)])[0]
    sl = (slice(margin, margin + w), slice(margin, margin + w))
    assert np.abs(win[sl] - full[np.ix_(ys, xs)][sl]).max() <= 1e-15 * np.abs(full).max()
