"""The paper's own cell (§2.3): the side-heated square cavity (hot left wall,
cold right wall, adiabatic top and bottom, all no-slip), validated by what the
physics fixes without outside reference values: at steady state the heat that
enters through the hot wall leaves through the cold wall and equals the
volume-averaged horizontal heat flux (the global Nusselt number of the
library), and the Nusselt number converges at second order in the grid."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP64 = 0


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_03160_gb300 import tlbm

    tlbm.lib()
    return tlbm


def _wall_nusselt(T, n):
    """Nusselt numbers of the hot (x = -1/2, T = +1/2) and cold (x = n - 1/2,
    T = -1/2) walls from a second-order one-sided gradient through the wall
    value and the first two nodes (distances 0, 1/2, 3/2 from the wall)."""
    dh = (-8 * 0.5 + 9 * T[:, 0] - T[:, 1]) / 3.0
    dc = -(-8 * -0.5 + 9 * T[:, -1] - T[:, -2]) / 3.0
    return -n * dh.mean(), -n * dc.mean()


def test_side_heated_cavity_heat_balance_and_convergence(T):
    out = {}
    for n, steps in ((65, 200000), (129, 400000)):
        g = T.Sim(n, n, lattice=0, Ra=1e5, Pr=0.71, Ma=0.1, precision=FP64, walls=1)
        g.init(1, 0.0)
        g.step(steps - 20000)
        nu0 = g.nusselt()
        g.step(20000)
        nu = g.nusselt()
        assert abs(nu - nu0) < 1e-6 * nu, (n, nu0, nu)  # steady
        hot, cold = _wall_nusselt(g.macros()["T"].cpu().numpy(), n)
        assert abs(hot - cold) < 1e-9 * hot, (n, hot, cold)  # point symmetry of the cavity
        out[n] = (nu, hot)
        g.close()
    gap = {n: abs(h - nu) / nu for n, (nu, h) in out.items()}
    # the heat through the walls equals the volume-averaged flux, to the wall
    # gradient's discretisation error, which shrinks at least 4x per doubling
    assert gap[65] < 3e-3 and gap[129] < 5e-4 and gap[129] < gap[65] / 4, gap
    # grid convergence of the global Nusselt number
    assert abs(out[65][0] - out[129][0]) < 0.01 * out[129][0], out
    assert out[129][0] > 4.0  # a convection-dominated flow at Ra = 1e5
