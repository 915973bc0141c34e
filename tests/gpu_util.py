"""Shared helpers of the GPU parity tests (inputs from workloads, references from the oracle)."""
import numpy as np

from paper_2203_11938_gb300 import workloads as W

MAT = np.array([1.0e3, 0.3, 1.0e-4, 0.1])


def to_cuda(a, dtype):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def to_np(t):
    return t.detach().double().cpu().numpy()


def make_batch(sheets, *, steps, dt, precision, tol, max_iter=5000, ckpt=0, exec_mode="graph", eta=1e-3, poll=16,
               precond="block", schedule=-1, warm=False):
    from paper_2203_11938_gb300 import sim

    meshes = [(s.rest, s.tris, s.pinned) for s in sheets]
    return sim.ClothBatch(meshes, steps=steps, dt=dt, precision=precision, cg_tol=tol, cg_max_iter=max_iter,
                          checkpoint_every=ckpt, clamp_eta=eta, exec_mode=exec_mode, cg_poll_every=poll,
                          precond=precond, cg_schedule=schedule, cg_warm_start=warm)


def oracle_sims(oracle, sheets):
    return [oracle.OracleSim(s.rest, s.tris, s.pinned) for s in sheets]


def split(arr, sizes, axis=0):
    out, off = [], 0
    for n in sizes:
        out.append(np.take(arr, np.arange(off, off + n), axis=axis))
        off += n
    return out


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def sheets_mixed(seed=3):
    """Three sheets of different (ragged) sizes and materials."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for N, pin in ((5, "top2"), (9, "top"), (13, "corners")):
        rest, tris = W.grid_mesh(N)
        out.append(W.Sheet(N, rest, tris, W.pins(N, pin), W.sample_material(rng), None))
    return out


def max_entry_err(a, b):
    """Largest entry-wise difference, relative to the largest entry of the reference: a
    localised error in a few entries shows here even where the norm of the whole field
    hides it."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
