"""Checkpoint and resume (tlbm_save / tlbm_load): a run resumed from a file
continues bitwise as the uninterrupted run, for every storage precision, both
streaming schemes and both wall configurations; mismatched handles and damaged
files are refused."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

D2, D3 = 0, 1
FP64, FP32, FP16, BF16 = 0, 1, 2, 3


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_03160_gb300 import tlbm

    tlbm.lib()
    return tlbm


CASES = [
    (D2, (129, 67, 1), FP32, {}),
    (D2, (129, 67, 1), BF16, {}),  # the staged kernel
    (D2, (96, 40, 1), FP16, {"walls": 1}),
    (D3, (37, 21, 19), FP16, {"streaming": 1}),
    (D3, (37, 21, 19), FP64, {}),
]


@pytest.mark.parametrize("lattice,shape,prec,kw", CASES)
def test_resume_is_bitwise(T, tmp_path, lattice, shape, prec, kw):
    args = dict(lattice=lattice, Ra=1e6, Pr=0.71, Ma=0.1, precision=prec, **kw)
    a = T.Sim(*shape, **args)
    a.init(3, 1e-3)
    a.step(37)
    path = tmp_path / "state.ckpt"
    a.save(path)
    a.step(21)
    b = T.Sim(*shape, **args)
    b.load(path)
    assert b.status()[1] == 37
    b.step(21)
    (fa, ga), (fb, gb) = a.get_populations(), b.get_populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert a.status() == b.status() == (False, 58)
    assert a.nusselt() == b.nusselt()
    q = 14 if lattice == D2 else 26
    head = path.stat().st_size - 8 * q * shape[0] * shape[1] * shape[2]
    assert 64 <= head <= 1024
    a.close()
    b.close()


def test_resume_across_streaming_schemes(T, tmp_path):
    args = dict(lattice=D2, Ra=1e6, Pr=0.71, Ma=0.1, precision=FP32)
    a = T.Sim(161, 83, **args)
    a.init(4, 1e-3)
    a.step(25)
    path = tmp_path / "pull.ckpt"
    a.save(path)
    a.step(10)
    b = T.Sim(161, 83, streaming=1, **args)
    b.load(path)
    b.step(10)
    (fa, ga), (fb, gb) = a.get_populations(), b.get_populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    a.close()
    b.close()


def test_load_refuses_mismatch_and_damage(T, tmp_path):
    args = dict(lattice=D2, Pr=0.71, Ma=0.1, precision=FP32)
    a = T.Sim(65, 33, Ra=1e5, **args)
    a.init(1, 1e-3)
    a.step(3)
    path = tmp_path / "a.ckpt"
    a.save(path)
    for other in (T.Sim(65, 33, Ra=2e5, **args), T.Sim(65, 35, Ra=1e5, **args),
                  T.Sim(65, 33, Ra=1e5, lattice=D2, Pr=0.71, Ma=0.1, precision=FP16),
                  T.Sim(65, 33, Ra=1e5, walls=1, **args)):
        with pytest.raises(T.TlbmError) as ei:
            other.load(path)
        assert ei.value.code == T.TLBM_ERR_ARG
        other.close()
    raw = path.read_bytes()
    for bad, data in (("short", raw[:-8]), ("long", raw + b"\0" * 8), ("magic", b"X" + raw[1:])):
        p = tmp_path / f"{bad}.ckpt"
        p.write_bytes(data)
        with pytest.raises(T.TlbmError) as ei:
            a.load(p)
        assert ei.value.code == T.TLBM_ERR_ARG, bad
    with pytest.raises(T.TlbmError) as ei:
        a.load(tmp_path / "missing.ckpt")
    assert ei.value.code == T.TLBM_ERR_ARG
    # the handle still works: the good file loads and steps
    a.load(path)
    assert a.status() == (False, 3)
    a.close()
