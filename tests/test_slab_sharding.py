"""Slab sharding of one tensor (the multi-GPU form of the sweep) on the CPU:
world-size-2 gloo process groups, each rank holding a contiguous slab of Y along
one observed letter and running the real planner and sweep driver (plan.cpp,
compiled into the host test double) on its slab.  Factors that do not hold the
split letter are updated from num/den all-reduced over the slabs (nef_numden,
nef_apply_update); the others are updated locally.  The assembled factors must
match the single-process FP64 oracle fit of the whole tensor (Algorithm 1)."""
import ctypes
import os
import socket
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CASES = [
    ("ir,jr,kr->ijk", dict(i=9, j=6, k=7, r=3), "i", True),
    ("ir,jr,kr->ijk", dict(i=5, j=6, k=11, r=2), "k", False),
    ("ia,ja,ab,kb,lb->ijkl", dict(i=4, j=7, k=3, l=5, a=2, b=3), "j", True),
]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem(model_str, dims, masked):
    sys.path.insert(0, ROOT)
    from oracle import OracleModel
    m = OracleModel(model_str, dims)
    import zlib
    rng = np.random.default_rng(zlib.crc32(f"{model_str}{masked}".encode()))  # same draw in every process
    fs = [rng.uniform(0.3, 1.7, size=m.factor_shape(l)) for l in range(m.n_factors)]
    y = rng.poisson(np.einsum(model_str, *fs)).astype(np.float64)
    mask = (rng.random(m.y_shape) > 0.25).astype(np.uint8) if masked else None
    return m, y, mask, fs


def _rank_main(rank, world, port, model_str, dims, letter, masked, iters, outdir):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(HERE, "hostcheck"))
    import torch
    import torch.distributed as dist
    import build as hostcheck_build
    from paper_2602_02759_gb300._nef import Options, split_model
    from paper_2602_02759_gb300.slab import slab_bounds, slab_sweeps

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        lib = ctypes.CDLL(hostcheck_build.LIB)
        vp = ctypes.c_void_p
        lib.nef_plan.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.POINTER(Options),
                                 ctypes.POINTER(vp)]
        lib.nef_update.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.POINTER(vp), ctypes.c_double, ctypes.c_double]
        lib.nef_numden.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.POINTER(vp), ctypes.c_double, ctypes.c_double,
                                   vp, vp]
        lib.nef_apply_update.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp), vp, vp, ctypes.c_double,
                                         ctypes.c_double]
        lib.nef_plan_destroy.argtypes = [vp]
        lib.nef_last_error.restype = ctypes.c_char_p
        m, y, mask, fs = _problem(model_str, dims, masked)
        obs, lat, terms = split_model(model_str)
        ax = obs.index(letter)
        lo, hi = slab_bounds(dims[letter], world, rank)
        sl = [slice(None)] * len(obs)
        sl[ax] = slice(lo, hi)
        y_s = np.ascontiguousarray(y[tuple(sl)])
        m_s = None if mask is None else np.ascontiguousarray(mask[tuple(sl)])
        local = [letter in t for t in terms]
        work = []
        for t, f in zip(terms, fs):
            if letter in t:
                fsl = [slice(None)] * len(t)
                fsl[t.index(letter)] = slice(lo, hi)
                work.append(np.ascontiguousarray(f[tuple(fsl)]))
            else:
                work.append(f.copy())
        sdims = dict(dims)
        sdims[letter] = hi - lo
        shapes = (ctypes.c_int64 * len(obs))(*[sdims[c] for c in obs])
        ranks = (ctypes.c_int64 * max(1, len(lat)))(*[sdims[c] for c in lat])
        o = Options()
        lib.nef_default_options(ctypes.byref(o))
        o.precision = 2  # NEF_FP64
        h = vp()
        assert lib.nef_plan(model_str.encode(), shapes, len(obs), ranks, len(lat), ctypes.byref(o),
                            ctypes.byref(h)) == 0, lib.nef_last_error()

        def facs():
            arr = (vp * len(work))()
            for k, f in enumerate(work):
                arr[k] = f.ctypes.data
            return arr

        mp = None if m_s is None else m_s.ctypes.data

        class Ops:
            def update(self, l):
                assert lib.nef_update(h, l, y_s.ctypes.data, mp, facs(), 1.0, 0.0) == 0, lib.nef_last_error()

            def numden(self, l):
                num = np.empty_like(work[l])
                den = np.empty_like(work[l])
                assert lib.nef_numden(h, l, y_s.ctypes.data, mp, facs(), 1.0, 0.0, num.ctypes.data,
                                      den.ctypes.data) == 0, lib.nef_last_error()
                return num, den

            def apply_update(self, l, num, den):
                assert lib.nef_apply_update(h, l, facs(), num.ctypes.data, den.ctypes.data, 1.0, 0.0) == 0, \
                    lib.nef_last_error()

        def allreduce(a):
            dist.all_reduce(torch.from_numpy(a), op=dist.ReduceOp.SUM)

        slab_sweeps(Ops(), local, iters, allreduce)
        lib.nef_plan_destroy(h)
        for k, f in enumerate(work):
            np.save(os.path.join(outdir, f"r{rank}_f{k}.npy"), f)
    finally:
        dist.destroy_process_group()


def test_slab_bounds_partition():
    from paper_2602_02759_gb300.slab import slab_bounds
    for n in (1, 2, 7, 10, 512):
        for world in (1, 2, 3, 8):
            if world > n:
                continue
            b = [slab_bounds(n, world, r) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in b]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1


@pytest.mark.parametrize("model_str,dims,letter,masked", CASES)
def test_slab_sharded_fit_matches_single_process_oracle(model_str, dims, letter, masked, tmp_path):
    sys.path.insert(0, os.path.join(HERE, "hostcheck"))
    import build as hostcheck_build
    import torch.multiprocessing as mp
    from paper_2602_02759_gb300._nef import split_model
    from paper_2602_02759_gb300.slab import slab_bounds
    hostcheck_build.build()
    iters, world = 3, 2
    mp.start_processes(_rank_main, args=(world, _free_port(), model_str, dims, letter, masked, iters, str(tmp_path)),
                       nprocs=world, join=True, start_method="spawn")
    m, y, mask, fs = _problem(model_str, dims, masked)
    ref = m.fit(y, mask, fs, 1.0, 0.0, iters)
    _, _, terms = split_model(model_str)
    for k, t in enumerate(terms):
        parts = [np.load(tmp_path / f"r{r}_f{k}.npy") for r in range(world)]
        if letter in t:
            got = np.concatenate(parts, axis=t.index(letter))
        else:
            np.testing.assert_array_equal(parts[0], parts[1])  # replicas stay identical
            got = parts[0]
        np.testing.assert_allclose(got, ref[k], rtol=1e-10, err_msg=f"factor {t}")
    for r in range(world):
        lo, hi = slab_bounds(dims[letter], world, r)
        assert hi > lo
