"""FP64 CPU oracle of the phi-SfT cloth step and its adjoint (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
The C++ source (``cloth_oracle.cpp``) is a plain, slow FP64 restatement of
Sec. 3.1 (Eq. 3-5) with forward-mode AD of the two element energies; it shares
no code with the CUDA library.

Arrays crossing this wrapper are numpy float64, AoS ``[n][3]`` per state.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cloth_oracle.cpp")
_LIB = os.path.join(_HERE, "libcloth_oracle.so")
_lib = None
ETA = 1e-3  # default smooth clamp of the membrane geometric stiffness, eps = ETA * Y (reading R6)
PRECOND = 1  # default CG preconditioner: 3x3 block Jacobi (0: scalar Jacobi)

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (portable flags, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_create.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _ip, _u8p, ctypes.POINTER(ctypes.c_void_p)]
        lib.oracle_create.restype = ctypes.c_int
        lib.oracle_destroy.argtypes = [ctypes.c_void_p]
        lib.oracle_num_hinges.argtypes = [ctypes.c_void_p]
        lib.oracle_num_hinges.restype = ctypes.c_int
        lib.oracle_hinges.argtypes = [ctypes.c_void_p, _ip, _dp, _dp]
        lib.oracle_mass.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp]
        lib.oracle_energy_forces.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
        lib.oracle_energy_forces.restype = ctypes.c_double
        lib.oracle_hessian_dense.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, _dp, _dp]
        lib.oracle_third.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, _dp, _dp, _dp, _dp]
        lib.oracle_membrane_element.argtypes = [_dp, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
        lib.oracle_membrane_element.restype = ctypes.c_int
        lib.oracle_dihedral.argtypes = [_dp]
        lib.oracle_dihedral.restype = ctypes.c_double
        lib.oracle_system_dense.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, _dp, _dp, _dp]
        lib.oracle_system_matvec.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp,
                                             _dp, _dp, _dp, _dp]
        lib.oracle_forward.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp,
                                       _ip, _ip]
        lib.oracle_forward.restype = ctypes.c_int
        lib.oracle_backward.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp,
                                        _dp, _dp, _dp, _dp, _ip, _ip]
        lib.oracle_backward.restype = ctypes.c_int
        lib.oracle_loss_l2.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
        lib.oracle_loss_l2.restype = ctypes.c_double
        lib.oracle_loss_pinhole.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
        lib.oracle_loss_pinhole.restype = ctypes.c_double
        _lib = lib
    return _lib


def _d(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class OracleSim:
    """One cloth sheet: rest mesh, triangles, pinned mask (Sec. 3.1)."""

    def __init__(self, rest, tris, pinned=None):
        lib = _load()
        self.rest = _f64(rest).reshape(-1, 3)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
        self.n = self.rest.shape[0]
        self.m = self.tris.shape[0]
        pin = np.zeros(self.n, np.uint8) if pinned is None else np.ascontiguousarray(pinned, dtype=np.uint8)
        self.pinned = pin
        h = ctypes.c_void_p()
        rc = lib.oracle_create(self.n, _d(self.rest), self.m, self.tris.ctypes.data_as(_ip),
                               pin.ctypes.data_as(_u8p), ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"oracle_create failed with code {rc}")
        self._h = h
        self._lib = lib

    def __del__(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.oracle_destroy(self._h)
            self._h = None

    # -- topology / mass
    def hinges(self):
        ne = self._lib.oracle_num_hinges(self._h)
        v = np.zeros((ne, 4), np.int32)
        w = np.zeros(ne)
        th = np.zeros(ne)
        self._lib.oracle_hinges(self._h, v.ctypes.data_as(_ip), _d(w), _d(th))
        return v, w, th

    def mass(self, rho):
        out = np.zeros(self.n)
        self._lib.oracle_mass(self._h, float(rho), _d(out))
        return out

    # -- element-level quantities
    def energy_forces(self, material, x):
        mat = _f64(material)
        x = _f64(x)
        fm = np.zeros((self.n, 3))
        fb = np.zeros((self.n, 3))
        E = self._lib.oracle_energy_forces(self._h, _d(mat), _d(x), _d(fm), _d(fb))
        return E, fm, fb

    def hessian_dense(self, material, x, eta=ETA):
        N = 3 * self.n
        H = np.zeros((N, N))
        self._lib.oracle_hessian_dense(self._h, _d(_f64(material)), float(eta), _d(_f64(x)), _d(H))
        return H

    def third(self, material, x, a, b, eta=ETA):
        out = np.zeros((self.n, 3))
        self._lib.oracle_third(self._h, _d(_f64(material)), float(eta), _d(_f64(x)), _d(_f64(a)), _d(_f64(b)), _d(out))
        return out

    def system_dense(self, material, dt, gravity, x, v, F=None, eta=ETA):
        N = 3 * self.n
        A = np.zeros((N, N))
        b = np.zeros(N)
        Fp = None if F is None else _f64(F)
        self._lib.oracle_system_dense(self._h, _d(_f64(material)), float(eta), float(dt), _d(_f64(gravity)), _d(_f64(x)),
                                      _d(_f64(v)), _d(Fp), _d(A), _d(b))
        return A, b

    def system_matvec(self, material, dt, gravity, x, v, F, p, eta=ETA):
        """(A p, b) of one step at (x, v) with external force F (any size)."""
        y = np.zeros((self.n, 3))
        b = np.zeros((self.n, 3))
        Fp = None if F is None else _f64(F)
        self._lib.oracle_system_matvec(self._h, _d(_f64(material)), float(eta), float(dt), _d(_f64(gravity)),
                                       _d(_f64(x)), _d(_f64(v)), _d(Fp), _d(_f64(p)), _d(y), _d(b))
        return y, b

    # -- trajectory
    def forward(self, material, x0, v0, forces, *, dt, steps, tol, max_iter, gravity, eta=ETA, precond=PRECOND,
                force_mode=0, air_density=0.0, wind=None):
        """force_mode 0: forces [N] added to f; 1: velocity increments [m/s] added to the
        free vertices' velocities before each step.  air_density > 0 with wind (3,):
        quadratic air drag of the relative wind on every free vertex."""
        tx = np.zeros((steps + 1, self.n, 3))
        tv = np.zeros((steps + 1, self.n, 3))
        iters = np.zeros(steps, np.int32)
        st = ctypes.c_int(0)
        Fp = None if forces is None else _f64(forces, (steps, self.n, 3))
        self._lib.oracle_forward(self._h, _d(_f64(material)), float(eta), int(precond), float(dt), int(steps), float(tol), int(max_iter),
                                 _d(_f64(gravity)), _d(_f64(x0, (self.n, 3))), _d(_f64(v0, (self.n, 3))), _d(Fp),
                                 int(force_mode), float(air_density), _d(None if wind is None else _f64(wind)),
                                 _d(tx), _d(tv), iters.ctypes.data_as(_ip), ctypes.byref(st))
        return tx, tv, iters, st.value

    def backward(self, material, traj_x, traj_v, dL_dx, *, dt, steps, tol, max_iter, gravity, eta=ETA,
                 precond=PRECOND, forces=None, force_mode=0, air_density=0.0, wind=None):
        """forces, force_mode, air_density, wind: as given to forward (the forces are read
        in mode 1 only).  The result adds "wind" = dL/dw."""
        gw = np.zeros(3)
        Fp = None if forces is None else _f64(forces, (steps, self.n, 3))
        gm = np.zeros(4)
        gF = np.zeros((steps, self.n, 3))
        gx0 = np.zeros((self.n, 3))
        gv0 = np.zeros((self.n, 3))
        iters = np.zeros(steps, np.int32)
        st = ctypes.c_int(0)
        self._lib.oracle_backward(self._h, _d(_f64(material)), float(eta), int(precond), float(dt), int(steps), float(tol), int(max_iter),
                                  _d(_f64(gravity)), _d(_f64(traj_x)), _d(_f64(traj_v)), _d(Fp), int(force_mode),
                                  float(air_density), _d(None if wind is None else _f64(wind)), _d(_f64(dL_dx)),
                                  _d(gm), _d(gF), _d(gx0), _d(gv0), _d(gw), iters.ctypes.data_as(_ip), ctypes.byref(st))
        return dict(material=gm, forces=gF, x0=gx0, v0=gv0, wind=gw, cg_iters=iters, status=st.value)


def membrane_element(rest, x, Y, nu):
    lib = _load()
    rest = _f64(rest)
    x = _f64(x)
    E = ctypes.c_double()
    g = np.zeros(9)
    H = np.zeros(81)
    rc = lib.oracle_membrane_element(_d(rest), _d(x), float(Y), float(nu), ctypes.byref(E), _d(g), _d(H))
    if rc != 0:
        raise ValueError("degenerate rest triangle")
    return E.value, g, H.reshape(9, 9)


def dihedral(x12):
    return _load().oracle_dihedral(_d(_f64(x12)))


def loss_l2(traj, target):
    traj = _f64(traj)
    target = _f64(target)
    steps = traj.shape[0] - 1
    n = traj.shape[1]
    g = np.zeros_like(traj)
    L = _load().oracle_loss_l2(n, steps, _d(traj), _d(target), _d(g))
    return L, g


def loss_pinhole(traj, target_uv, cam):
    traj = _f64(traj)
    target_uv = _f64(target_uv)
    steps = traj.shape[0] - 1
    n = traj.shape[1]
    g = np.zeros_like(traj)
    L = _load().oracle_loss_pinhole(n, steps, _d(_f64(cam)), _d(traj), _d(target_uv), _d(g))
    return L, g
