"""Write the stored oracle values of the full-size parity tests (tests/golden/*.npz).

Calls only the FP64 oracle (``oracle/``) and the seeded input generators
(``paper_2203_11938_gb300/workloads.py``); nothing here touches the CUDA library.
Each case runs the oracle's forward trajectory and its adjoint (Sec. 3.1, Eq. 3-5 and
the implicit differentiation of every solve) on inputs rounded to float, exactly as the
FP32 path receives them, and stores the values the GPU tests compare entry by entry:

  batch_largest, batch_slowest
      sheets 93 (64 x 64) and 220 (61 x 61) of the 256-sheet batch (seed 1), 100 steps of
      1/30 s, two top corners pinned, no external force; loss L = sum_{t>=1} |x_t - X|^2
      (X: the template); oracle CG tol 1e-10.
  batch_n16, batch_n22, batch_n30, batch_n38, batch_n42, batch_n46, batch_n54, batch_n56
      one sheet of each of those grid sides from the same batch (workloads.
      BATCH_GOLDEN_CLASSES), the same run.
  grid100_segment
      the 100 x 100 sheet of the pinhole workload, its first 30 steps (one checkpoint
      segment) with the smooth wind; loss = pinhole reprojection against the template's
      tracks (workloads.template_tracks); oracle CG tol 1e-9.
  grid100_full
      the same sheet over the workload's whole trajectory (300 steps, ten checkpoint
      segments of 30); loss and tolerance as above.
  grid256_segment
      the 256 x 256 sheet with four corners pinned, its first 20 steps (the workload's
      first checkpoint segment) with the smooth wind (the oracle needs about 75 s per
      solve at this size); loss L = sum_{t>=1} |x_t - X|^2; oracle CG tol 1e-8.
      Per-vertex arrays are stored for every 5th vertex (all norms are of the full
      arrays).
  grid256_two_segments
      the same over its first two checkpoint segments (40 steps).

Run: python tests/golden/make_fullsize_goldens.py [case ...]   (hours of CPU time; each
case runs in its own process, all cases in parallel).
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

CASES = ("batch_largest", "batch_slowest", "batch_n16", "batch_n22", "batch_n30", "batch_n38", "batch_n42",
         "batch_n46", "batch_n54", "batch_n56", "grid100_segment", "grid100_full", "grid256_segment",
         "grid256_two_segments")
# the 256 x 256 workload checkpoints every 20 steps: its stored run is one whole segment
GRID256_STEPS = 20


def f32r(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _case_inputs(case):
    from paper_2203_11938_gb300 import workloads as W

    if case.startswith("batch_"):
        cfg = W.config4()
        name = case.split("_", 1)[1]
        k = W.BATCH_GOLDEN_SHEETS.get(name, W.BATCH_GOLDEN_CLASSES.get(name))
        s = cfg.sheets[k]
        return dict(sheet=s, index=k, steps=cfg.steps, dt=cfg.dt, forces=None, loss="l2", tol=1e-10, stride=1)
    if case == "grid100_segment":
        cfg = W.config3(steps=30)
        s = cfg.sheets[0]
        return dict(sheet=s, index=0, steps=30, dt=cfg.dt, forces=s.forces[:30], loss="pinhole", tol=1e-9,
                    stride=1, camera=cfg.camera)
    if case == "grid100_full":
        cfg = W.config3()
        s = cfg.sheets[0]
        return dict(sheet=s, index=0, steps=cfg.steps, dt=cfg.dt, forces=s.forces[:cfg.steps], loss="pinhole",
                    tol=1e-9, stride=1, camera=cfg.camera)
    if case.startswith("grid256_"):
        T = GRID256_STEPS if case == "grid256_segment" else 2 * GRID256_STEPS
        cfg = W.config5(steps=T)
        s = cfg.sheets[0]
        return dict(sheet=s, index=0, steps=T, dt=cfg.dt, forces=s.forces[:T], loss="l2",
                    tol=1e-8, stride=5)
    raise ValueError(case)


def run_case(case):
    import oracle
    from paper_2203_11938_gb300 import workloads as W

    c = _case_inputs(case)
    s, T, dt = c["sheet"], c["steps"], c["dt"]
    mat, x0 = f32r(s.material), f32r(s.rest)
    F = None if c["forces"] is None else f32r(c["forces"])
    o = oracle.OracleSim(s.rest, s.tris, s.pinned)
    t0 = time.time()
    kw = dict(dt=dt, steps=T, tol=c["tol"], max_iter=40000, gravity=W.GRAVITY)
    tx, tv, it_f, st_f = o.forward(mat, x0, np.zeros_like(x0), F, **kw)
    t1 = time.time()
    if c["loss"] == "pinhole":
        uv = W.template_tracks(s.rest, T)
        L, dL = oracle.loss_pinhole(tx, uv, c["camera"])
    else:
        L, dL = oracle.loss_l2(tx, np.broadcast_to(x0, tx.shape))
    g = o.backward(mat, tx, tv, dL, forces=F, **kw)
    t2 = time.time()
    sel = np.arange(0, s.n, c["stride"])
    rows = sorted({0, T // 2, T - 1})
    out = {
        "case": case, "sheet_index": c["index"], "N": s.N, "steps": T, "dt": dt, "oracle_tol": c["tol"],
        "loss_kind": c["loss"], "material": mat, "vertex_sample": sel,
        "x_mid": tx[T // 2][sel], "x_final": tx[T][sel], "v_final": tv[T][sel], "loss": L,
        "g_material": g["material"], "g_x0": g["x0"][sel], "g_v0": g["v0"][sel],
        "g_x0_norm": np.linalg.norm(g["x0"]), "g_v0_norm": np.linalg.norm(g["v0"]),
        "cg_iters_forward": it_f, "cg_iters_adjoint": g["cg_iters"],
        "status": np.array([st_f, g["status"]]), "seconds": np.array([t1 - t0, t2 - t1]),
    }
    if F is not None:
        out["g_forces_rows"] = np.array(rows)
        out["g_forces"] = g["forces"][rows][:, sel]
        out["g_forces_norm"] = np.linalg.norm(g["forces"])
    np.savez_compressed(os.path.join(HERE, f"{case}.npz"), **out)
    summary = {"case": case, "N": s.N, "steps": T, "loss": float(L), "g_material": g["material"].tolist(),
               "cg_iters_forward_total": int(it_f.sum()), "cg_iters_adjoint_total": int(g["cg_iters"].sum()),
               "status": [int(st_f), int(g["status"])], "seconds": [round(t1 - t0, 1), round(t2 - t1, 1)]}
    print(json.dumps(summary), flush=True)
    return summary


def main():
    cases = sys.argv[1:] or list(CASES)
    for cs in cases:
        if cs not in CASES:
            raise SystemExit(f"unknown case {cs}; cases: {', '.join(CASES)}")
    import oracle

    oracle.build()
    with mp.get_context("spawn").Pool(len(cases)) as pool:
        pool.map(run_case, cases)


if __name__ == "__main__":
    main()
