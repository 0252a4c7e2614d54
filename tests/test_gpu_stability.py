"""The linear-stability tool (Sec. III) on the GPU against the oracle's
amplification matrix, for the Mach-1 and Mach-3 states of Fig. 2."""
import numpy as np
import pytest

from oracle import fdlb
from oracle.stability import amplification_matrix
from paper_1106_0785_gb300 import stability

pytestmark = pytest.mark.gpu

DX, DT = 1e-3, 1e-5


def _rates(over):
    s = np.full(16, 1e5)
    s[:4] = 0
    for k, v in over.items():
        s[k - 1] = v  # the paper's 1-based index
    return s


CASES = {"a": ((2.0, 2.0, 0.0, 2.0), {}), "b": ((2.0, 6.0, 0.0, 2.0), {9: 1e3})}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("version", [1, 3])
def test_amplification_matrix_matches_the_oracle(cuda, case, version):
    (rho, ux, uy, T), over = CASES[case]
    s = _rates(over)
    kd, G = stability.amplification(s, rho, ux, uy, T, dx=DX, dy=DX, dt=DT, n=64, version=version)
    p = fdlb.Params(nx=4, ny=4, dx=DX, dy=DX, dt=DT, s=s, version=version)
    for k, g in zip(kd, G):
        want = amplification_matrix(p, rho, ux, uy, T, k / DX, 0.0)
        assert np.abs(g - want).max() < 1e-6 * max(1.0, np.abs(want).max()), (k, np.abs(g - want).max())


def test_growth_along_y_matches_x_for_a_state_moving_along_y(cuda):
    """Rotating the state and the axis by 90 degrees leaves the spectrum: the
    tool's y path agrees with its x path."""
    s = _rates({9: 1e3, 10: 1e3})  # the pair of moments 9, 10 rotate into each other
    gx = stability.max_growth(s, 2.0, 6.0, 0.0, 2.0, dx=DX, dy=DX, dt=DT, n=64, axis=0)
    gy = stability.max_growth(s, 2.0, 0.0, 6.0, 2.0, dx=DX, dy=DX, dt=DT, n=64, axis=1)
    assert abs(gx - gy) < 1e-5  # the central differences resolve G to ~1e-6
