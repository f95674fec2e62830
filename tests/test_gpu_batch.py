"""Batched ensemble: every instance of a batch evolves exactly as the same cell
stepped on its own, for every batch variant and with CUDA-graph step blocks;
small instances also match the FP64 oracle."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_03160_gb300 import tlbm

    tlbm.lib()
    return tlbm


def _draws(n, sizes, seed=4, lattice=0):
    out = []
    for N, Ra, Pr, s in inputs.ensemble_draws(seed, n, sizes=sizes, log_ra=(5.0, 7.0)):
        out.append((N, N + 3, N - 2 if lattice else 1, Ra, Pr, 0.1, s))
    return out


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_batch_equals_single_instances(T, prec):
    inst = _draws(7, (33, 65, 129))
    b = T.Batch(inst, lattice=0, precision=prec)
    b.init(1e-3)
    b.step(37)  # a graph block of 16 steps, twice, plus single launches
    singles = []
    for nx, ny, nz, Ra, Pr, Ma, seed in inst:
        s = T.Sim(nx, ny, nz, lattice=0, Ra=Ra, Pr=Pr, Ma=Ma, precision=prec)
        v, form, bx, by = b.variant[:4]
        s.set_variant(v, form, bx, by)
        s.init(seed, 1e-3)
        s.step(37)
        singles.append(s.get_populations())
    for k in range(len(inst)):
        fb, gb = b.get_populations(k)
        fs, gs = singles[k]
        # same arithmetic in another kernel: equal up to the compiler's
        # multiply-add contraction choices (one rounding of the storage type)
        tol = {0: 1e-13, 1: 1e-6, 2: 1e-3, 3: 4e-3}[prec]
        assert np.abs(fb - fs).max() <= tol and np.abs(gb - gs).max() <= tol, k


def test_batch_3d_and_oracle(T, O):
    inst = [(9, 11, 7, 1e5, 0.71, 0.1, 3), (13, 9, 10, 3e5, 7.0, 0.1, 4), (17, 8, 9, 1e6, 0.71, 0.1, 5)]
    b = T.Batch(inst, lattice=1, precision=0)
    b.init(1e-3)
    b.step(20)
    for k, (nx, ny, nz, Ra, Pr, Ma, seed) in enumerate(inst):
        o = O.Sim(nx, ny, nz, lattice=1, Ra=Ra, Pr=Pr, Ma=Ma)
        o.init(seed, 1e-3)
        o.step(20)
        fb, gb = b.get_populations(k)
        fo, go = o.get_populations()
        assert np.abs(fb - fo).max() < 1e-12 and np.abs(gb - go).max() < 1e-12


def test_batch_variants_and_autotune_keep_state(T):
    inst = _draws(9, (129, 257))
    b = T.Batch(inst, lattice=0, precision=1)
    b.init(1e-3)
    b.step(6)
    before = [b.get_populations(k) for k in (0, 4, 8)]
    b.autotune(3)
    after = [b.get_populations(k) for k in (0, 4, 8)]
    for (f0, g0), (f1, g1) in zip(before, after):
        assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
    ref = None
    for vec, form, bx, by, gs in ((4, 2, 32, 1, 16), (2, 2, 64, 2, 0), (4, 1, 32, 4, 4), (0, 0, 0, 0, 2)):
        c = T.Batch(inst, lattice=0, precision=1)
        c.set_variant(vec, form, bx, by, gs)
        c.init(1e-3)
        c.step(11)
        pops = [c.get_populations(k) for k in (0, 4, 8)]
        if ref is None:
            ref = pops
        else:
            for (f0, g0), (f1, g1) in zip(ref, pops):
                assert np.abs(f0 - f1).max() < 2e-6 and np.abs(g0 - g1).max() < 2e-6
        c.close()


def test_batch_reductions_and_status(T):
    inst = _draws(5, (65, 129))
    b = T.Batch(inst, lattice=0, precision=1)
    b.init(1e-3)
    b.step(10)
    nus = b.nusselt()
    assert len(nus) == 5 and all(np.isfinite(nus))
    assert b.status() == [False] * 5
    for k in range(5):
        assert abs(T.tlbm_nusselt(b.instance(k)) - nus[k]) == 0.0
    assert b.launches >= 10


@pytest.mark.parametrize("lattice,prec", [(0, 1), (0, 2), (1, 3), (0, 0)])
def test_persistent_batch_equals_flattened_launches(T, lattice, prec):
    """The persistent form (one cooperative launch for many steps, a bounded grid
    barrier between steps) computes exactly what the flattened per-step launches
    compute, for step counts that end on either buffer and span several
    launches."""
    inst = _draws(6, (33, 65, 97), lattice=lattice)
    ref = T.Batch(inst, lattice=lattice, precision=prec)
    per = T.Batch(inst, lattice=lattice, precision=prec)
    v = ref.variant
    per.set_variant(v[0], v[1], v[2], v[3], 0)
    per.set_persistent(7)
    for b in (ref, per):
        b.init(1e-3)
    for n in (1, 9, 20):
        ref.step(n)
        per.step(n)
        for k in (0, 3, 5):
            (fa, ga), (fb, gb) = ref.get_populations(k), per.get_populations(k)
            assert np.array_equal(fa, fb) and np.array_equal(ga, gb), (n, k)
        assert per.status() == [False] * 6
    # 30 steps: the first persistent launch of 7 steps, then ...: launches counted per launch
    assert per.launches == 1 + 2 + 3
    ref.close()
    per.close()


def test_autotune_cache_reuses_the_tuned_shape(T):
    inst = _draws(5, (129, 257), seed=9)
    a = T.Batch(inst, lattice=0, precision=1)
    a.init(1e-3)
    a.autotune(2)
    tuned = a.variant[:4]
    b = T.Batch(inst, lattice=0, precision=1)
    b.init(1e-3)
    l0 = b.launches
    b.autotune(-1)  # cached: no timing launches
    assert b.variant[:4] == tuned and b.launches == l0
    a.close()
    b.close()


@pytest.mark.parametrize("lattice,prec", [(0, 1), (0, 2), (0, 3), (1, 1), (1, 2)])
def test_batch_pipelined_rows_equal_one_row(T, lattice, prec):
    """Two rows per thread (software-pipelined body) in the flattened batch
    launch give bitwise the states of one row per thread, for odd row counts
    and step counts spanning a graph block; the persistent form switches back to
    one row and still agrees."""
    inst = _draws(5, (33, 65, 97), seed=6, lattice=lattice)
    a = T.Batch(inst, lattice=lattice, precision=prec)
    b = T.Batch(inst, lattice=lattice, precision=prec)
    vec = {(0, 1): 4, (0, 2): 8, (0, 3): 4, (1, 1): 1, (1, 2): 1}[(lattice, prec)]
    for x in (a, b):
        x.set_variant(vec, 2, 32, 2, 16)
    a.set_rows(1)
    b.set_rows(2)
    assert (a.rows, b.rows) == (1, 2)
    for x in (a, b):
        x.init(1e-3)
        x.step(37)
    for k in range(len(inst)):
        (fa, ga), (fb, gb) = a.get_populations(k), b.get_populations(k)
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), k
    b.set_persistent(8)
    for x in (a, b):
        x.step(16)
    for k in range(len(inst)):
        (fa, ga), (fb, gb) = a.get_populations(k), b.get_populations(k)
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), k
    a.close()
    b.close()


_STAGED_CELLS = {
    # ragged rows, rows cut into several segments (600 > 8 x 64, 300 > 4 x 64)
    0: [(33, 36, 1, 3e5, 0.71, 0.1, 21), (65, 40, 1, 1e6, 7.0, 0.1, 22), (300, 23, 1, 2e5, 0.71, 0.1, 23),
        (600, 9, 1, 5e5, 7.0, 0.1, 24)],
    1: [(9, 11, 7, 1e5, 0.71, 0.1, 25), (17, 8, 9, 3e5, 7.0, 0.1, 26), (300, 5, 4, 1e6, 0.71, 0.1, 27)],
}


@pytest.mark.parametrize("lattice,prec,nc", [(0, 1, 4), (0, 1, 8), (0, 2, 4), (0, 2, 8), (0, 3, 8), (1, 1, 7),
                                             (1, 2, 4), (1, 2, 7), (1, 3, 7)])
def test_staged_batch_equals_single_staged_cells(T, lattice, prec, nc):
    """The staged batch form (one producer/consumer pipeline over the tiles of
    every instance) steps each instance bitwise as the single-cell staged kernel
    steps that cell alone: ragged rows, rows cut into several segments, 3D
    instances, 37 steps (two CUDA-graph blocks and single launches), and for
    16-bit storage the stochastic rounding keyed by each instance's own step
    count."""
    inst = _STAGED_CELLS[lattice]
    b = T.Batch(inst, lattice=lattice, precision=prec)
    b.set_staged(nc)
    assert b.staged[0] == nc and b.staged[1] >= 2
    b.init(1e-3)
    b.step(37)
    assert b.status() == [False] * len(inst)
    for k, (nx, ny, nz, Ra, Pr, Ma, seed) in enumerate(inst):
        s = T.Sim(nx, ny, nz, lattice=lattice, Ra=Ra, Pr=Pr, Ma=Ma, precision=prec)
        s.set_staged(0, 0)
        s.init(seed, 1e-3)
        s.step(37)
        (fb, gb), (fs, gs) = b.get_populations(k), s.get_populations()
        assert np.array_equal(fb, fs) and np.array_equal(gb, gs), k
        s.close()
    # an explicit register-kernel shape turns the staged form off
    b.set_variant(0, 0, 0, 0, 16)
    assert b.staged == (0, 0, 0)
    b.close()


def test_staged_batch_rejects_what_it_cannot_run(T):
    inst = _STAGED_CELLS[0][:2]
    b = T.Batch(inst, lattice=0, precision=0)  # FP64
    with pytest.raises(T.TlbmError) as ei:
        b.set_staged(8)
    assert ei.value.code == T.TLBM_ERR_UNSUPPORTED
    c = T.Batch(inst, lattice=0, precision=2)
    with pytest.raises(T.TlbmError) as ei:
        c.set_staged(7)  # 4 or 8 in 2D
    assert ei.value.code == T.TLBM_ERR_ARG
    c.set_persistent(4)
    with pytest.raises(T.TlbmError) as ei:
        c.set_staged(8)
    assert ei.value.code == T.TLBM_ERR_UNSUPPORTED
    b.close()
    c.close()


def test_staged_batch_wait_times_out_and_recovers(T):
    inst = _STAGED_CELLS[0]
    b = T.Batch(inst, lattice=0, precision=2)
    b.set_staged(8)
    b.set_wait_limit(0)
    b.init(1e-3)
    b.step(6)
    with pytest.raises(T.TlbmError) as ei:
        b.status()
    assert ei.value.code == T.TLBM_ERR_TIMEOUT
    b.set_wait_limit(0.5)
    b.init(1e-3)
    b.step(20)
    assert b.status() == [False] * len(inst)
    ref = T.Batch(inst, lattice=0, precision=2)
    ref.set_staged(8)
    ref.init(1e-3)
    ref.step(20)
    for k in range(len(inst)):
        (fa, ga), (fb, gb) = b.get_populations(k), ref.get_populations(k)
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), k
    b.close()
    ref.close()
