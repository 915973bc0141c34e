"""Python binding of the C-ABI cloth library (argument marshalling only).

Every step of the simulator and its adjoint runs in the CUDA kernels of
``_lib/libcloth_sim.so``; this module only checks tensors, passes their device
pointers and the current CUDA stream through ctypes, and wraps the pair
forward/backward as a ``torch.autograd.Function``.  PyTorch provides device memory
and streams.  There is no CPU path: without the built library or a GPU every call
raises.

Layouts follow ``include/cloth_sim.h``: per-vertex tensors are ``[N_total, 3]`` in
the packed user order (sheet 0's vertices, then sheet 1's, ...); trajectories are
``[steps + 1, N_total, 3]``; forces ``[steps, N_total, 3]``; materials
``[count, 4]`` = (Y, nu, k_b, rho).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcloth_sim.so")

FP32, FP64 = 0, 1
EXEC_PLAIN, EXEC_GRAPH = 0, 1
STATUS_CG_MAXITER, STATUS_INDEFINITE, STATUS_NONFINITE, STATUS_PINNED_VELOCITY_NONZERO = 1, 2, 4, 8

# exported names declared in include/cloth_sim.h
EXPORTS = (
    "cloth_default_opts", "cloth_mesh_create", "cloth_mesh_destroy", "cloth_mesh_info", "cloth_batch_create",
    "cloth_batch_destroy", "cloth_batch_info", "cloth_forward", "cloth_backward", "cloth_loss_l2",
    "cloth_loss_pinhole", "cloth_stats", "cloth_internal_forces", "cloth_system_dense", "cloth_spmv",
    "cloth_third_contraction", "cloth_last_error", "cloth_matrix_info", "cloth_time_kernel", "cloth_loss_l2_static",
    "cloth_sheet_iterations", "cloth_kernel_bytes", "cloth_set_wind", "cloth_wind_gradient",
    "cloth_image_energy_scratch", "cloth_image_energy",
)


class ClothOpts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("steps", ctypes.c_int32),
        ("dt", ctypes.c_double),
        ("cg_tol", ctypes.c_double),
        ("cg_max_iter", ctypes.c_int32),
        ("checkpoint_every", ctypes.c_int32),
        ("gravity", ctypes.c_double * 3),
        ("clamp_eta", ctypes.c_double),
        ("exec", ctypes.c_int32),
        ("cg_poll_every", ctypes.c_int32),
        ("precond", ctypes.c_int32),
        ("cg_schedule", ctypes.c_int32),
        ("cg_handover", ctypes.c_int32),
        ("force_mode", ctypes.c_int32),
        ("air_density", ctypes.c_double),
        ("cg_warm_start", ctypes.c_int32),
    ]


_lib = None
_vp = ctypes.c_void_p


def load_library(path: str = LIB_PATH):
    """Load the shared library (no GPU needed to load it)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2203_11938_gb300.build.build()")
    lib = ctypes.CDLL(path)
    lib.cloth_default_opts.argtypes = [ctypes.POINTER(ClothOpts)]
    lib.cloth_default_opts.restype = None
    lib.cloth_last_error.restype = ctypes.c_char_p
    lib.cloth_mesh_create.argtypes = [_vp, ctypes.c_int32, _vp, ctypes.c_int32, _vp, ctypes.POINTER(_vp)]
    lib.cloth_mesh_destroy.argtypes = [_vp]
    lib.cloth_mesh_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int32)]
    lib.cloth_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(ClothOpts),
                                       ctypes.POINTER(_vp)]
    lib.cloth_batch_destroy.argtypes = [_vp]
    lib.cloth_batch_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_size_t)]
    lib.cloth_forward.argtypes = [_vp] * 8
    lib.cloth_backward.argtypes = [_vp] * 8
    lib.cloth_loss_l2.argtypes = [_vp] * 6
    lib.cloth_loss_pinhole.argtypes = [_vp] * 7
    lib.cloth_stats.argtypes = [_vp] * 5
    lib.cloth_matrix_info.argtypes = [_vp] * 5
    lib.cloth_sheet_iterations.argtypes = [_vp, ctypes.c_int32, _vp, _vp]
    lib.cloth_kernel_bytes.argtypes = [_vp, ctypes.c_int32, _vp]
    lib.cloth_set_wind.argtypes = [_vp, _vp]
    lib.cloth_image_energy_scratch.argtypes = [ctypes.c_int32] * 4
    lib.cloth_image_energy_scratch.restype = ctypes.c_size_t
    lib.cloth_image_energy.argtypes = [ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32,
                                       _vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                       _vp]
    lib.cloth_wind_gradient.argtypes = [_vp, _vp, _vp]
    lib.cloth_time_kernel.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp]
    lib.cloth_internal_forces.argtypes = [_vp] * 6
    lib.cloth_system_dense.argtypes = [_vp] * 8
    lib.cloth_spmv.argtypes = [_vp] * 7
    lib.cloth_third_contraction.argtypes = [_vp] * 7
    lib.cloth_loss_l2_static.argtypes = [ctypes.c_int32, _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp, _vp,
                                         _vp, _vp, _vp]
    for name in EXPORTS:
        f = getattr(lib, name)
        if name not in ("cloth_default_opts", "cloth_last_error"):
            f.restype = ctypes.c_int
    _lib = lib
    return lib


class ClothError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        msg = _lib.cloth_last_error().decode(errors="replace")
        raise ClothError(f"{what} failed ({rc}): {msg}")


def default_opts() -> ClothOpts:
    o = ClothOpts()
    load_library().cloth_default_opts(ctypes.byref(o))
    return o


def _ptr(t):
    return None if t is None else _vp(t.data_ptr())


class Mesh:
    """A sheet's template mesh (host arrays: rest [n,3] float64, tris [m,3] int32, pinned [n])."""

    def __init__(self, rest, tris, pinned=None):
        lib = load_library()
        self.rest = np.ascontiguousarray(rest, np.float64).reshape(-1, 3)
        self.tris = np.ascontiguousarray(tris, np.int32).reshape(-1, 3)
        self.pinned = None if pinned is None else np.ascontiguousarray(pinned, np.uint8)
        h = _vp()
        _check(lib.cloth_mesh_create(self.rest.ctypes.data, self.rest.shape[0], self.tris.ctypes.data,
                                     self.tris.shape[0], None if self.pinned is None else self.pinned.ctypes.data,
                                     ctypes.byref(h)), "cloth_mesh_create")
        self._h = h

    def info(self):
        n, m, e = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.cloth_mesh_info(self._h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(e)), "cloth_mesh_info")
        return n.value, m.value, e.value

    def __del__(self):
        if getattr(self, "_h", None) is not None and self._h.value and _lib is not None:
            _lib.cloth_mesh_destroy(self._h)
            self._h = None


class ClothBatch:
    """A batch of sheets stepped together (``cloth_batch_create``)."""

    def __init__(self, meshes, *, steps, dt, precision="f32", cg_tol=1e-6, cg_max_iter=2000, checkpoint_every=0,
                 gravity=(0.0, 0.0, -9.8), clamp_eta=1e-3, exec_mode="graph", cg_poll_every=16, precond="block",
                 cg_schedule=-1, cg_handover=0, force_mode="force", air_density=0.0, cg_warm_start=False):
        import torch

        if not torch.cuda.is_available():
            raise ClothError("a CUDA device is required (there is no CPU path)")
        lib = load_library()
        self.meshes = [m if isinstance(m, Mesh) else Mesh(*m) for m in meshes]
        o = default_opts()
        o.precision = FP64 if precision == "f64" else FP32
        o.steps = int(steps)
        o.dt = float(dt)
        o.cg_tol = float(cg_tol)
        o.cg_max_iter = int(cg_max_iter)
        o.checkpoint_every = int(checkpoint_every)
        for k in range(3):
            o.gravity[k] = float(gravity[k])
        o.clamp_eta = float(clamp_eta)
        o.exec = EXEC_GRAPH if exec_mode == "graph" else EXEC_PLAIN
        o.cg_poll_every = int(cg_poll_every)
        o.precond = 1 if precond == "block" else 0
        o.cg_schedule = int(cg_schedule)
        o.cg_handover = int(cg_handover)
        o.force_mode = {"force": 0, "velocity": 1}[force_mode]
        o.air_density = float(air_density)
        o.cg_warm_start = 1 if cg_warm_start else 0
        self.opts = o
        self.steps = int(steps)
        self.dtype = torch.float64 if precision == "f64" else torch.float32
        arr = (_vp * len(self.meshes))(*[m._h for m in self.meshes])
        h = _vp()
        _check(lib.cloth_batch_create(arr, len(self.meshes), ctypes.byref(o), ctypes.byref(h)), "cloth_batch_create")
        self._h = h
        nt, cnt, ws = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t()
        _check(lib.cloth_batch_info(h, ctypes.byref(nt), ctypes.byref(cnt), ctypes.byref(ws)), "cloth_batch_info")
        self.total_vertices, self.count, self.workspace_bytes = nt.value, cnt.value, ws.value
        self.sheet_sizes = [m.rest.shape[0] for m in self.meshes]

    def __del__(self):
        if getattr(self, "_h", None) is not None and self._h.value and _lib is not None:
            _lib.cloth_batch_destroy(self._h)
            self._h = None

    # -------------------------------------------------------------- helpers
    def _stream(self):
        import torch

        return _vp(torch.cuda.current_stream().cuda_stream)

    def _t(self, t, shape, name, dtype=None):
        import torch

        if t is None:
            return None
        dtype = dtype or self.dtype
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ClothError(f"{name} must be a CUDA tensor")
        if t.dtype != dtype:
            raise ClothError(f"{name} must have dtype {dtype}, got {t.dtype}")
        if tuple(t.shape) != tuple(shape):
            raise ClothError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ClothError(f"{name} must be contiguous")
        return t

    def _new(self, *shape, dtype=None):
        import torch

        return torch.empty(*shape, dtype=dtype or self.dtype, device="cuda")

    # -------------------------------------------------------------- entry points
    def forward(self, material, x0, v0, forces=None):
        import torch

        N, S, T = self.total_vertices, self.count, self.steps
        self._t(material, (S, 4), "material")
        self._t(x0, (N, 3), "x0")
        self._t(v0, (N, 3), "v0")
        self._t(forces, (T, N, 3), "forces")
        traj = self._new(T + 1, N, 3)
        status = torch.zeros(S, dtype=torch.int32, device="cuda")
        self._fwd_forces = forces  # the backward's recompute reads it again
        _check(_lib.cloth_forward(self._h, _ptr(material), _ptr(x0), _ptr(v0), _ptr(forces), _ptr(traj),
                                  _ptr(status), self._stream()), "cloth_forward")
        return traj, status

    def backward(self, dL_dx, want=("material", "forces", "x0", "v0")):
        import torch

        N, S, T = self.total_vertices, self.count, self.steps
        self._t(dL_dx, (T + 1, N, 3), "dL_dx")
        out = {
            "material": self._new(S, 4) if "material" in want else None,
            "forces": self._new(T, N, 3) if "forces" in want else None,
            "x0": self._new(N, 3) if "x0" in want else None,
            "v0": self._new(N, 3) if "v0" in want else None,
        }
        status = torch.zeros(S, dtype=torch.int32, device="cuda")
        _check(_lib.cloth_backward(self._h, _ptr(dL_dx), _ptr(out["material"]), _ptr(out["forces"]),
                                   _ptr(out["x0"]), _ptr(out["v0"]), _ptr(status), self._stream()), "cloth_backward")
        out["status"] = status
        return out

    def loss_l2(self, traj, target, want_grad=True):
        import torch

        N, S, T = self.total_vertices, self.count, self.steps
        self._t(traj, (T + 1, N, 3), "traj")
        self._t(target, (T + 1, N, 3), "target")
        loss = torch.empty(S, dtype=torch.float64, device="cuda")
        grad = self._new(T + 1, N, 3) if want_grad else None
        _check(_lib.cloth_loss_l2(self._h, _ptr(traj), _ptr(target), _ptr(loss), _ptr(grad), self._stream()),
               "cloth_loss_l2")
        return loss, grad

    def loss_pinhole(self, traj, target_uv, camera, want_grad=True):
        import torch

        N, S, T = self.total_vertices, self.count, self.steps
        self._t(traj, (T + 1, N, 3), "traj")
        self._t(target_uv, (T + 1, N, 2), "target_uv")
        cam = (ctypes.c_double * 4)(*[float(c) for c in camera])
        loss = torch.empty(S, dtype=torch.float64, device="cuda")
        grad = self._new(T + 1, N, 3) if want_grad else None
        _check(_lib.cloth_loss_pinhole(self._h, _ptr(traj), _ptr(target_uv), cam, _ptr(loss), _ptr(grad),
                                       self._stream()), "cloth_loss_pinhole")
        return loss, grad

    def stats(self):
        f, b, r, n = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.cloth_stats(self._h, ctypes.byref(f), ctypes.byref(b), ctypes.byref(r), ctypes.byref(n)),
               "cloth_stats")
        return {"fwd_cg_iters": f.value, "bwd_cg_iters": b.value, "recompute_cg_iters": r.value,
                "kernel_launches": n.value}

    PHASES = {"forward": 0, "adjoint": 1, "recompute": 2}

    def sheet_iterations(self, phase="forward"):
        """Per-sheet CG iterations of the last call of `phase`: (largest single solve,
        sum over solves), each a numpy array [count]."""
        import numpy as np

        mx = np.zeros(self.count, np.int32)
        tot = np.zeros(self.count, np.int64)
        _check(_lib.cloth_sheet_iterations(self._h, self.PHASES[phase], mx.ctypes.data_as(_vp),
                                           tot.ctypes.data_as(_vp)), "cloth_sheet_iterations")
        return mx, tot

    def matrix_info(self):
        r, b, s, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(_lib.cloth_matrix_info(self._h, ctypes.byref(r), ctypes.byref(b), ctypes.byref(s), ctypes.byref(c)),
               "cloth_matrix_info")
        return {"rows": r.value, "blocks": b.value, "stored_blocks": s.value, "cg_schedule": c.value}

    KERNELS = {"spmv": 0, "cg_update": 1, "assemble": 2, "elem_tri": 3, "elem_hinge": 4, "cg_solve": 5}

    def time_kernel(self, name, reps=20):
        ms = ctypes.c_double()
        _check(_lib.cloth_time_kernel(self._h, self.KERNELS[name], int(reps), ctypes.byref(ms), self._stream()),
               "cloth_time_kernel")
        return ms.value

    def set_wind(self, wind):
        """Per-sheet wind velocity [count, 3] (device, batch precision) or None; kept by
        reference and read by the following forward and backward calls."""
        if wind is not None:
            self._t(wind, (self.count, 3), "wind")
        self._wind = wind
        _check(_lib.cloth_set_wind(self._h, _ptr(wind)), "cloth_set_wind")

    def wind_gradient(self):
        """dL/dw of the last backward, [count, 3]."""
        g = self._new(self.count, 3)
        _check(_lib.cloth_wind_gradient(self._h, _ptr(g), self._stream()), "cloth_wind_gradient")
        return g

    def kernel_bytes(self, name):
        """Algorithmic bytes of one launch of the kernel time_kernel(name) times."""
        b = ctypes.c_int64()
        _check(_lib.cloth_kernel_bytes(self._h, self.KERNELS[name], ctypes.byref(b)), "cloth_kernel_bytes")
        return b.value

    def internal_forces(self, material, x):
        N, S = self.total_vertices, self.count
        self._t(material, (S, 4), "material")
        self._t(x, (N, 3), "x")
        fm, fb = self._new(N, 3), self._new(N, 3)
        _check(_lib.cloth_internal_forces(self._h, _ptr(material), _ptr(x), _ptr(fm), _ptr(fb), self._stream()),
               "cloth_internal_forces")
        return fm, fb

    def system_dense(self, material, x, v, F=None):
        N, S = self.total_vertices, self.count
        self._t(material, (S, 4), "material")
        self._t(x, (N, 3), "x")
        self._t(v, (N, 3), "v")
        self._t(F, (N, 3), "F")
        total = sum((3 * n) ** 2 for n in self.sheet_sizes)
        A = self._new(total)
        b = self._new(N, 3)
        _check(_lib.cloth_system_dense(self._h, _ptr(material), _ptr(x), _ptr(v), _ptr(F), _ptr(A), _ptr(b),
                                       self._stream()), "cloth_system_dense")
        blocks, off = [], 0
        for n in self.sheet_sizes:
            blocks.append(A[off:off + 9 * n * n].view(3 * n, 3 * n))
            off += 9 * n * n
        return blocks, b

    def spmv(self, material, x, v, p):
        N, S = self.total_vertices, self.count
        for t, nm in ((x, "x"), (v, "v"), (p, "p")):
            self._t(t, (N, 3), nm)
        self._t(material, (S, 4), "material")
        y = self._new(N, 3)
        _check(_lib.cloth_spmv(self._h, _ptr(material), _ptr(x), _ptr(v), _ptr(p), _ptr(y), self._stream()),
               "cloth_spmv")
        return y

    def third(self, material, x, a, b):
        N, S = self.total_vertices, self.count
        for t, nm in ((x, "x"), (a, "a"), (b, "b")):
            self._t(t, (N, 3), nm)
        self._t(material, (S, 4), "material")
        out = self._new(N, 3)
        _check(_lib.cloth_third_contraction(self._h, _ptr(material), _ptr(x), _ptr(a), _ptr(b), _ptr(out),
                                            self._stream()), "cloth_third_contraction")
        return out


def _autograd_function():
    import torch

    class ClothTrajectory(torch.autograd.Function):
        """traj = PS rollout (Eq. 1) of a batch; backward = the library's adjoint.

        apply(batch, material [S,4], x0 [N,3], v0 [N,3], forces [T,N,3] or None) -> traj [T+1,N,3].
        Gradients flow to material (Y, k_b, rho; nu gets 0), x0, v0 and forces.
        """

        @staticmethod
        def forward(ctx, batch, material, x0, v0, forces):
            traj, status = batch.forward(material.contiguous(), x0.contiguous(), v0.contiguous(),
                                         None if forces is None else forces.contiguous())
            ctx.batch = batch
            ctx.has_forces = forces is not None
            ctx.status = status
            return traj

        @staticmethod
        def backward(ctx, g):
            out = ctx.batch.backward(g.contiguous())
            gF = out["forces"] if ctx.has_forces else None
            return None, out["material"], out["x0"], out["v0"], gF

    return ClothTrajectory


_CT = None


def image_energy(x, tris, uv, tex, camera, image, mask, want_grad=True, want_render=False):
    """Image energy E = E_p + 0.5 E_s of one sheet against one frame (cloth_image_energy):
    x [n, 3], uv [n, 2], tex [Ht, Wt, 3], image [H, W, 3], mask [H, W] (CUDA float64
    tensors), tris [m, 3] int (host), camera (f, cx, cy, cz).  Returns (E [1], dE/dx [n, 3]
    or None, rendered image or None, silhouette or None)."""
    import numpy as np
    import torch

    # shapes first (the kernels index x as [n][3], uv as [n][2], tex as [Ht][Wt][3],
    # image as [H][W][3] with n, H, W taken from x and mask), then devices and types
    tr = np.ascontiguousarray(np.asarray(tris, np.int32))
    if tr.ndim != 2 or tr.shape[1] != 3:
        raise ClothError(f"tris must have shape [m, 3], got {tuple(tr.shape)}")
    for t, name in ((x, "x"), (uv, "uv"), (tex, "tex"), (image, "image"), (mask, "mask")):
        if not isinstance(t, torch.Tensor):
            raise ClothError(f"{name} must be a torch tensor")
    if x.ndim != 2 or x.shape[1] != 3:
        raise ClothError(f"x must have shape [n, 3], got {tuple(x.shape)}")
    n = x.shape[0]
    if tuple(uv.shape) != (n, 2):
        raise ClothError(f"uv must have shape {(n, 2)}, got {tuple(uv.shape)}")
    if tex.ndim != 3 or tex.shape[2] != 3:
        raise ClothError(f"tex must have shape [Ht, Wt, 3], got {tuple(tex.shape)}")
    if mask.ndim != 2:
        raise ClothError(f"mask must have shape [H, W], got {tuple(mask.shape)}")
    if tuple(image.shape) != tuple(mask.shape) + (3,):
        raise ClothError(f"image must have shape {tuple(mask.shape) + (3,)}, got {tuple(image.shape)}")
    for t, name in ((x, "x"), (uv, "uv"), (tex, "tex"), (image, "image"), (mask, "mask")):
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ClothError(f"{name}: expected a contiguous CUDA float64 tensor")
    load_library()
    m = tr.shape[0]
    H, W = mask.shape
    scratch = torch.empty(int(_lib.cloth_image_energy_scratch(n, m, W, H)) // 8 + 1, dtype=torch.float64,
                          device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.empty(n, 3, dtype=torch.float64, device="cuda") if want_grad else None
    img = torch.empty(H, W, 3, dtype=torch.float64, device="cuda") if want_render else None
    sil = torch.empty(H, W, dtype=torch.float64, device="cuda") if want_render else None
    cam = (ctypes.c_double * 4)(*[float(c) for c in camera])
    stream = torch.cuda.current_stream().cuda_stream
    _check(_lib.cloth_image_energy(n, m, tr.ctypes.data_as(_vp), _ptr(x), _ptr(uv), tex.shape[1], tex.shape[0],
                                   _ptr(tex), cam, W, H, _ptr(image), _ptr(mask), _ptr(scratch), _ptr(E), _ptr(g),
                                   _ptr(img), _ptr(sil), _vp(stream)), "cloth_image_energy")
    return E, g, img, sil


def cloth_trajectory(batch, material, x0, v0, forces=None):
    """Differentiable rollout through ``ClothTrajectory`` (see its docstring)."""
    global _CT
    if _CT is None:
        _CT = _autograd_function()
    return _CT.apply(batch, material, x0, v0, forces)
