"""In-place (AA-pattern) streaming: one population buffer, steps alternating
between a half that reads and writes every node's own slots and a half that
reads from and pushes to the neighbours.  Checked against the FP64 CPU oracle
on tiny and ragged grids with every wall / periodic combination (after odd
and even step counts, so both storage orders are read back), and bitwise
against the two-buffer pull kernels (the collision is the same code)."""
import numpy as np
import pytest

import inputs
from test_gpu_parity import D2, D3, EDGE_CASES, FP16, FP32, FP64, BF16, TOL1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_03160_gb300 import tlbm

    tlbm.lib()
    return tlbm


# compiled in-place variants: (vec, form), form 1 = general MRT, 2 = TRT evaluation
AA_VARIANTS = {
    (D2, FP32): [(4, 2), (1, 2), (4, 1)], (D2, FP16): [(4, 2), (1, 2), (4, 1)], (D2, BF16): [(4, 2), (1, 2), (4, 1)],
    (D2, FP64): [(2, 2), (2, 1)],
    (D3, FP32): [(1, 2), (2, 2), (1, 1)], (D3, FP16): [(2, 2), (1, 2), (2, 1)], (D3, BF16): [(2, 2), (1, 2), (2, 1)],
    (D3, FP64): [(1, 2), (1, 1)],
}


@pytest.mark.parametrize("prec", [FP64, FP32, FP16, BF16])
@pytest.mark.parametrize("lattice,shape,walls,pm", EDGE_CASES)
def test_inplace_random_populations_match_oracle(T, O, prec, lattice, shape, walls, pm):
    nx, ny, nz = shape
    o = O.Sim(nx, ny, nz, lattice=lattice, Ra=1e5, Pr=0.71, Ma=0.1, walls=walls, periodic_mask=pm)
    qf, qg = (9, 5) if lattice == D2 else (19, 7)
    seed = 11 + 13 * lattice + 3 * walls + pm + 100 * prec + nx
    f = inputs.uniform_array(seed, (qf,) + o.shape, 0.02, 0.2)
    gg = inputs.uniform_array(seed + 1, (qg,) + o.shape, -0.1, 0.1)
    ref = None
    for vec, form in AA_VARIANTS[(lattice, prec)]:
        g = T.Sim(nx, ny, nz, lattice=lattice, Ra=1e5, Pr=0.71, Ma=0.1, precision=prec, walls=walls,
                  periodic_mask=pm, streaming=T.TLBM_STREAM_INPLACE)
        g.set_variant(vec, form)
        g.set_populations(f, gg)
        f0, g0 = g.get_populations()
        if ref is None:
            o.set_populations(f0, g0)
            ref = []
            for n in (1, 2, 1):  # after 1 (swapped order), 3 (swapped), 4 (natural) steps
                o.step(n)
                ref.append(o.get_populations())
        done = 0
        for (fo, go), n in zip(ref, (1, 2, 1)):
            g.step(n)
            done += n
            fg, ggg = g.get_populations()
            ef = np.abs(fg - fo).max() / np.abs(fo).max()
            eg = np.abs(ggg - go).max() / np.abs(go).max()
            assert ef < TOL1[prec] * done and eg < TOL1[prec] * done, (vec, form, done, ef, eg)
        g.close()


@pytest.mark.parametrize("lattice,shape,prec", [
    (D2, (301, 45, 1), FP32), (D2, (301, 45, 1), FP16), (D2, (130, 33, 1), BF16), (D2, (129, 65, 1), FP64),
    (D3, (77, 21, 13), FP32), (D3, (77, 21, 13), BF16), (D3, (40, 9, 11), FP16), (D3, (33, 12, 10), FP64)])
def test_inplace_equals_pull_bitwise(T, lattice, shape, prec):
    """Same collision code, same results: states, macros and Nusselt number of the
    in-place and the two-buffer runs agree exactly after odd and even step counts."""
    sims = [T.Sim(*shape, lattice=lattice, Ra=1e6, Pr=0.71, Ma=0.1, precision=prec, streaming=s)
            for s in (T.TLBM_STREAM_PULL, T.TLBM_STREAM_INPLACE)]
    for s in sims:
        # the register kernel with the same nodes per thread on both sides
        s.set_variant(sims[1].variant[0], 2)
        s.init(5, 1e-3)
    for n in (1, 2, 5, 20, 37):
        for s in sims:
            s.step(n)
        (fa, ga), (fb, gb) = (s.get_populations() for s in sims)
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), n
        ma, mb = (s.macros() for s in sims)
        for k in ma:
            assert np.array_equal(ma[k].cpu().numpy(), mb[k].cpu().numpy()), (n, k)
        assert sims[0].nusselt() == sims[1].nusselt()
        assert sims[0].energy() == sims[1].energy()
    for s in sims:
        s.close()


def test_inplace_halves_memory_and_rejects_two_buffer_kernels(T):
    a = T.Sim(257, 129, lattice=D2, Ra=1e6, Pr=0.71, Ma=0.1, precision=FP32)
    b = T.Sim(257, 129, lattice=D2, Ra=1e6, Pr=0.71, Ma=0.1, precision=FP32, streaming=T.TLBM_STREAM_INPLACE)
    pop = 14 * 4 * 257 * 129
    assert a.nbytes - b.nbytes >= pop
    with pytest.raises(T.TlbmError) as ei:
        b.set_staged()
    assert ei.value.code == T.TLBM_ERR_UNSUPPORTED
    with pytest.raises(T.TlbmError) as ei:
        b.set_variant(4, 2, 32, 4, 2)
    assert ei.value.code == T.TLBM_ERR_UNSUPPORTED
    a.close()
    b.close()


def test_inplace_full_size_window(T):
    """8193^2 FP16 in place against the two-buffer run after 3 steps, on windows at
    the corners, the walls and the interior (the launch configuration the
    benchmark times)."""
    n = 8193
    outs = []
    for s in (T.TLBM_STREAM_PULL, T.TLBM_STREAM_INPLACE):
        g = T.Sim(n, n, lattice=D2, Ra=1e8, Pr=0.71, Ma=0.1, precision=FP16, streaming=s)
        g.set_variant(4, 2)
        g.init(2, 1e-3)
        g.step(3)
        outs.append([g.get_window(x, y, 0, 40, 24, 1) for x, y in ((0, 0), (n - 40, n - 24), (4000, 0), (0, 4100),
                                                                    (4090, 4090))])
        assert not g.status()[0]
        g.close()
    for (fa, ga), (fb, gb) in zip(*outs):
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
