"""Brute-force pin of the oracle's streaming and wall rules on tiny grids.

The oracle streams as a PULL (each node fetches f_i from x - e_i).  Here an
independent PUSH routine (each node sends f_i+ to x + e_i; what leaves the cell
bounces back at the node it came from, §2.2) is applied to the oracle's own
per-node collision; one oracle step must agree with it on random populations,
for every corner, edge and wall combination.
"""
import itertools

import numpy as np
import pytest

import inputs


def _push_step(O, sim, f, g, lattice, walls, periodic_mask, omega, Th=0.5, Tc=-0.5):
    ef = O.velocity_set(0 if lattice == 0 else 2)[0]
    eg = O.velocity_set(1 if lattice == 0 else 3)[0]
    of = O.velocity_set(0 if lattice == 0 else 2)[2]
    og = O.velocity_set(1 if lattice == 0 else 3)[2]
    qf, qg = len(ef), len(eg)
    spatial = f.shape[1:]
    dims = tuple(reversed(spatial))  # (nx, ny[, nz])
    D = len(dims)
    fpost = np.zeros_like(f)
    gpost = np.zeros_like(g)
    for idx in itertools.product(*[range(n) for n in spatial]):
        fo, go = sim.collide_node(f[(slice(None),) + idx], g[(slice(None),) + idx])
        fpost[(slice(None),) + idx] = fo
        gpost[(slice(None),) + idx] = go
    fn = np.full_like(f, np.nan)
    gn = np.full_like(g, np.nan)
    heat_axis = (1 if D == 2 else 2) if walls == 0 else 0
    for idx in itertools.product(*[range(n) for n in spatial]):
        c = list(reversed(idx))  # (x, y[, z])
        for pops, post, new, e, opp, thermal in ((f, fpost, fn, ef, of, False),
                                                 (g, gpost, gn, eg, og, True)):
            for i in range(len(e)):
                d = [c[a] + e[i][a] for a in range(D)]
                crossed = None
                for a in range(D):
                    if d[a] < 0 or d[a] >= dims[a]:
                        if periodic_mask & (1 << a):
                            d[a] %= dims[a]
                        else:
                            crossed = (a, d[a] >= dims[a])
                val = post[(i,) + idx]
                if crossed is None:
                    new[(i,) + tuple(reversed(d))] = val
                else:
                    if thermal and crossed[0] == heat_axis:
                        Tw = Tc if crossed[1] else Th
                        new[(opp[i],) + idx] = -val + omega * Tw
                    else:
                        new[(opp[i],) + idx] = val
    assert not np.isnan(fn).any() and not np.isnan(gn).any()
    return fn, gn


CASES = [
    (0, (3, 3, 1), 0, 0), (0, (4, 5, 1), 0, 0), (0, (5, 4, 1), 1, 0), (0, (4, 5, 1), 0, 1),
    (0, (5, 4, 1), 0, 2), (0, (3, 4, 1), 1, 3),
    (1, (5, 4, 3), 0, 0), (1, (3, 4, 5), 1, 0), (1, (4, 3, 3), 0, 1), (1, (3, 3, 4), 0, 6),
    (1, (4, 3, 3), 1, 5),
]


@pytest.mark.parametrize("lattice,shape,walls,pm", CASES)
def test_one_step_pull_equals_push(O, lattice, shape, walls, pm):
    nx, ny, nz = shape
    sim = O.Sim(nx, ny, nz, lattice=lattice, Ra=1e5, Pr=0.71, Ma=0.1, walls=walls,
                periodic_mask=pm)
    qf, qg = (9, 5) if lattice == 0 else (19, 7)
    sp = sim.shape
    seed = 100 + 7 * lattice + 13 * walls + pm
    f = inputs.uniform_array(seed, (qf,) + sp, 0.02, 0.2)
    g = inputs.uniform_array(seed + 1, (qg,) + sp, -0.1, 0.1)
    sim.set_populations(f, g)
    sim.step(1)
    fo, go = sim.get_populations()
    fp, gp = _push_step(O, sim, f, g, lattice, walls, pm, sim.derived()["omega"])
    assert np.abs(fo - fp).max() < 1e-15
    assert np.abs(go - gp).max() < 1e-15


def test_collision_is_local_and_step_counts(O):
    """A node's collision depends on its own populations only, and step(n)
    advances the step counter by n."""
    sim = O.Sim(4, 4, Ra=1e5, Pr=0.71, Ma=0.1)
    sim.init(1, 1e-3)
    f, g = sim.get_populations()
    a = sim.collide_node(f[:, 1, 2], g[:, 1, 2])
    f2 = f.copy()
    f2[:, 0, 0] *= 1.01
    b = sim.collide_node(f2[:, 1, 2], g[:, 1, 2])
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    sim.step(3)
    assert sim.time == 3
