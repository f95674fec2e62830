"""The cases of the bounds test: every step variant, storage precision and wall
configuration on small and ragged cells, the in-place scheme, the batched
ensemble (flattened, persistent and staged, 2D and 3D), the population transfers, checkpoints and
the reductions.  run() returns, per case, a digest of the final state and of
the reductions, and (with the bounds-checked library) the number of accesses
that left the population buffers.

Run as a script (python bounds_cases.py out.json) it loads the library the
environment selects, so that TLBM_DEBUG_BOUNDS=1 runs the cases on the
bounds-checked build in a process of its own."""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

D2, D3 = 0, 1
FP64, FP32, FP16, BF16 = 0, 1, 2, 3

# lattice, (nx, ny, nz), walls, periodic mask
SHAPES = [
    (D2, (3, 3, 1), 0, 0), (D2, (37, 9, 1), 0, 0), (D2, (131, 5, 1), 0, 1), (D2, (257, 4, 1), 1, 0),
    (D2, (6, 3, 1), 1, 3), (D3, (5, 4, 3), 0, 0), (D3, (35, 4, 3), 0, 0), (D3, (70, 3, 4), 0, 7),
    (D3, (4, 3, 3), 1, 5),
]
# (vec, form, rows) of every compiled two-buffer register variant
VARIANTS = {
    (D2, FP32): [(4, 2, 1), (2, 2, 1), (1, 2, 1), (4, 1, 1), (4, 2, 2), (4, 2, 4)],
    (D2, FP16): [(8, 2, 1), (4, 2, 1), (2, 2, 1), (8, 1, 1), (4, 2, 2), (8, 2, 4)],
    (D2, BF16): [(8, 2, 1), (4, 2, 1), (2, 2, 1), (8, 1, 1), (8, 2, 2), (4, 2, 4)],
    (D2, FP64): [(2, 2, 1), (1, 2, 1), (2, 1, 1)],
    (D3, FP32): [(4, 2, 1), (2, 2, 1), (1, 2, 1), (2, 1, 1), (1, 2, 2), (1, 2, 4)],
    (D3, FP16): [(4, 2, 1), (2, 2, 1), (1, 2, 1), (4, 1, 1), (1, 2, 2)],
    (D3, BF16): [(4, 2, 1), (2, 2, 1), (1, 2, 1), (4, 1, 1), (1, 2, 4)],
    (D3, FP64): [(1, 2, 1), (2, 2, 1), (1, 1, 1)],
}


def _digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(a.tobytes())
    return h.hexdigest()[:20]


def _violations(T, h):
    try:
        return T.tlbm_bounds_violations(h)
    except T.TlbmError as e:
        if e.code == T.TLBM_ERR_UNSUPPORTED:
            return None
        raise


def _finish(T, s, out, key):
    f, g = s.get_populations()
    nu = s.nusselt()
    ek, mass = s.energy()
    out[key] = {"hash": _digest(f, g), "red": [nu, ek, mass], "violations": _violations(T, s.h)}


def run(T, tmp_dir):
    out = {}
    for lattice, shape, walls, pm in SHAPES:
        kw = dict(lattice=lattice, Ra=1e5, Pr=0.71, Ma=0.1, walls=walls, periodic_mask=pm)
        for prec in (FP64, FP32, FP16, BF16):
            tag = f"{lattice}-{'x'.join(map(str, shape))}-w{walls}-p{pm}-q{prec}"
            kinds = [("reg",) + v for v in VARIANTS[(lattice, prec)]]
            if prec != FP64:
                kinds += [("staged", 16 // (4 if prec == FP32 else 2), 3), ("staged", 0, 0)]
            kinds += [("inplace",)]
            for kind in kinds:
                s = T.Sim(*shape, precision=prec, **kw,
                          streaming=T.TLBM_STREAM_INPLACE if kind[0] == "inplace" else T.TLBM_STREAM_PULL)
                if kind[0] == "reg":
                    s.set_variant(kind[1], kind[2], 0, 0, kind[3])
                elif kind[0] == "staged":
                    s.set_staged(kind[1], kind[2])
                s.init(5, 1e-3)
                s.step(7)
                _finish(T, s, out, f"{tag}-{'-'.join(map(str, kind))}")
                s.close()
        # transfers and checkpoints on the FP16 cell: set_populations, a
        # checkpoint round trip, initial fields
        s = T.Sim(*shape, precision=FP16, **kw)
        s.init(6, 1e-3)
        s.step(3)
        f, g = s.get_populations()
        s.set_populations(f, g)
        path = os.path.join(tmp_dir, f"c{lattice}{shape[0]}.ckpt")
        s.save(path)
        s.load(path)
        s.step(2)
        _finish(T, s, out, f"{lattice}-{'x'.join(map(str, shape))}-w{walls}-p{pm}-transfers")
        s.close()
    # the batched ensemble: flattened, persistent and staged (4 and the most consumer warps;
    # rows of the 300-node cell cut into two segments with 4 warps)
    inst2 = [(33, 33, 1, 1e5, 0.71, 0.1, 1), (65, 41, 1, 3e5, 7.0, 0.1, 2), (17, 17, 1, 1e6, 0.71, 0.1, 3),
             (300, 9, 1, 2e5, 7.0, 0.1, 4)]
    inst3 = [(9, 11, 7, 1e5, 0.71, 0.1, 5), (17, 8, 9, 3e5, 7.0, 0.1, 6), (300, 5, 4, 1e6, 0.71, 0.1, 7)]
    cases = [(D2, inst2, prec, mode) for prec in (FP32, FP16) for mode in ("flat", "persist", "staged4", "staged8")]
    cases += [(D3, inst3, FP16, mode) for mode in ("flat", "staged4", "staged7")]
    for lattice, inst, prec, mode in cases:
        b = T.Batch(inst, lattice=lattice, precision=prec)
        if mode == "persist":
            b.set_persistent(4)
        elif mode.startswith("staged"):
            b.set_staged(int(mode[len("staged"):]))
        b.init(1e-3)
        b.step(9)
        for k in range(len(inst)):
            f, g = b.get_populations(k)
            h = T.tlbm_batch_instance(b.b, k)
            out[f"batch-{lattice}-q{prec}-{mode}-{k}"] = {"hash": _digest(f, g), "red": [],
                                                          "violations": _violations(T, h)}
        b.close()
    return out


if __name__ == "__main__":
    from paper_2211_03160_gb300 import tlbm

    tlbm.lib()
    res = run(tlbm, os.path.dirname(os.path.abspath(sys.argv[1])))
    with open(sys.argv[1], "w") as fh:
        json.dump(res, fh)
