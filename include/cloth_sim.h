/*
 * cloth_sim.h - C ABI of the GB300 cloth simulator step and its adjoint.
 *
 * The library implements the differentiable physics simulator PS of phi-SfT
 * (Kairanda et al., CVPR 2022), Sec. 3.1 "Deformation Model":
 *   S_t = PS(S_{t-1}; phi_{t-1})                                       (Eq. 1)
 *   phi = {d, S, B, w, F}: density, stretching, bending, wind, per-step
 *         per-vertex corrective forces                                  (Eq. 2)
 *   d^2x/dt^2 = M^{-1} f(x, v), M lumped from density and area          (Eq. 3)
 *   implicit backward Euler, linearised:                                (Eq. 4-5)
 *       (M - h^2 K) dv = h (f + h K v),   v' = v + dv,   x' = x + h v'
 * and the gradient of a trajectory loss with respect to the material, the
 * per-step forces and the initial state by implicit differentiation of every
 * linear solve (Sec. 3.1, backward pass).  The paper leaves the elastic
 * energies open; this library uses an isotropic St. Venant-Kirchhoff membrane
 * on the Green strain (stretch stiffness Y [N/m], Poisson ratio nu) and a
 * dihedral-angle bending energy 1/2 k_b w_e (theta - theta_rest)^2 per interior
 * edge with w_e = 3 |e|^2 / (A_1 + A_2).  df/dv = 0 unless the optional air drag
 * (cloth_opts.air_density > 0) is on; its velocity Jacobian then enters Eq. 5.
 *
 * Conventions for every entry point:
 *   - Return value: CLOTH_OK (0) or a negative CLOTH_ERR_* code; on error a
 *     thread-local message is available from cloth_last_error().
 *   - "device" pointers are CUDA device (or managed) memory owned by the
 *     caller; the library never frees them.  "host" pointers are read during
 *     the call only.  The library owns only its handles and the workspace it
 *     allocates at cloth_batch_create (size: cloth_batch_info).
 *   - Floating-point device buffers have the batch precision: float for
 *     CLOTH_FP32, double for CLOTH_FP64.
 *   - Per-vertex arrays use the packed USER layout: the vertices of sheet 0,
 *     then sheet 1, ..., each vertex 3 consecutive values (x, y, z):
 *     [N_total][3].  Trajectories and forces stack steps in front:
 *     [steps + 1][N_total][3] and [steps][N_total][3].
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous with respect to the host unless stated otherwise.
 *   - Pinned vertices keep dv = 0 (kinematic pins): their velocity never
 *     changes, so with v0 = 0 they stay at x0; a nonzero v0 on a pinned vertex sets
 *     CLOTH_STATUS_PINNED_VELOCITY_NONZERO in its sheet's status word.
 */
#ifndef CLOTH_SIM_H
#define CLOTH_SIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define CLOTH_OK 0
#define CLOTH_ERR_INVALID_ARG (-1)    /* null pointer, bad size, bad option       */
#define CLOTH_ERR_NONMANIFOLD (-2)    /* edge in > 2 triangles or bad winding      */
#define CLOTH_ERR_DEGENERATE (-3)     /* zero-area rest triangle                   */
#define CLOTH_ERR_CUDA (-4)           /* a CUDA runtime call failed                */
#define CLOTH_ERR_OOM (-5)            /* workspace allocation failed               */
#define CLOTH_ERR_STATE (-6)          /* backward without a matching forward       */

/* ---- per-sheet status bits (device int32 per sheet, OR-ed over a call) ---- */
#define CLOTH_STATUS_CG_MAXITER 1     /* a solve stopped at cg_max_iter            */
#define CLOTH_STATUS_INDEFINITE 2     /* p^T A p <= 0 met inside CG                */
#define CLOTH_STATUS_NONFINITE 4      /* NaN/Inf in a CG scalar                    */
#define CLOTH_STATUS_PINNED_VELOCITY_NONZERO 8 /* cloth_forward: v0 is nonzero (or not
                                         finite) on a pinned vertex of the sheet.  Pins
                                         are kinematic (dv = 0), so such a vertex moves
                                         at its v0 for the whole trajectory instead of
                                         staying at x0; the run itself continues      */

/* ---- options ---- */
#define CLOTH_FP32 0
#define CLOTH_FP64 1

#define CLOTH_EXEC_PLAIN 0       /* host-driven CG loop, convergence polled per chunk */
#define CLOTH_EXEC_GRAPH 1       /* whole trajectory in one CUDA graph; CG loops are
                                    device-driven conditional WHILE nodes           */

typedef struct cloth_opts {
  int32_t precision;        /* CLOTH_FP32 or CLOTH_FP64                               */
  int32_t steps;            /* T >= 1 time steps per trajectory                       */
  double dt;                /* h > 0 [s]                                              */
  double cg_tol;            /* CG stops when |r|_2 <= cg_tol |b|_2 (per sheet)        */
  int32_t cg_max_iter;      /* >= 1                                                   */
  int32_t checkpoint_every; /* C: velocities and positions kept every C steps; the
                               backward recomputes each segment. 0 or >= steps: keep
                               the whole trajectory, no recompute                   */
  double gravity[3];        /* [m/s^2], e.g. {0, 0, -9.8}                             */
  double clamp_eta;         /* membrane geometric stiffness in the matrix uses the
                               smooth positive stress (S + (S^2 + (eta Y)^2 I)^1/2)/2;
                               0 = exact Hessian (may be indefinite)                 */
  int32_t exec;             /* CLOTH_EXEC_*                                           */
  int32_t cg_poll_every;    /* PLAIN mode: CG iterations between host polls (>= 1)    */
  int32_t precond;          /* CG preconditioner: CLOTH_PRECOND_JACOBI (scalar diagonal)
                               or CLOTH_PRECOND_BLOCK_JACOBI (3x3 block per vertex)   */
  int32_t cg_schedule;      /* CG kernel schedule, all with bitwise-identical results:
                               -1 = autotune at cloth_batch_create (times each schedule
                               on the batch's matrix, and the element kernels at 64,
                               128 and 256 threads per CTA; caches the choice in the
                               JSON file $CLOTH_TUNE_CACHE or
                               ~/.cache/cloth_sim/tune.json); an explicit schedule
                               keeps 128 threads per CTA for the element kernels;
                               0..31: bit 1 is always set (the direction update is
                               folded into the SpMV; a value without it means the same),
                               bit 0 = resident-CTA grid looping over rows, bit 2 =
                               per-sheet cluster solver for the sheets still iterating
                               at the hand-over point (every sheet of at most 8192
                               vertices, or 12288 where clusters of 16 CTAs can be
                               launched, gets one thread-block cluster), bit 3 (with
                               bit 2) = the on-chip variant of that solver for every
                               sheet whose matrix and vectors fit the shared memory of
                               at most 16 CTAs (the others keep the first variant),
                               bit 4 (with bit 2, without bit 3) = that solver with two
                               256-row work entries per CTA, clusters of up to 8 CTAs
                               and two CTAs per SM                                    */
  int32_t cg_handover;      /* with schedule bit 2: the device loop runs while more than
                               this many sheets are still iterating, then the per-sheet
                               solver finishes them (>= count: no loop at all);
                               0 = chosen by the autotuner (cg_schedule = -1: timed
                               whole solves of the loop alone and of hand-overs at
                               count/16 ... count), or every sheet (explicit schedule) */
  int32_t force_mode;       /* how the per-step per-vertex input F_t of cloth_forward
                               acts: CLOTH_FORCES_FORCE (a force [N] added to f, Eq. 3)
                               or CLOTH_FORCES_VELOCITY (a velocity increment [m/s]
                               added to the free vertices' velocities before step t,
                               the form the paper's implementation details give its
                               corrective forces, Sec. 3.4); the backward then returns dL/dF_t
                               in the same sense                                      */
  double air_density;       /* rho_air [kg/m^3] >= 0; > 0 adds the air drag of the
                               relative wind velocity d = w - v on every free vertex,
                               f = rho_air A s(d) d with its lumped rest area A and
                               s(d) = (|d|^2 + (1e-3 m/s)^2)^1/2, implicit through
                               df/dv in the step matrix (Eq. 5); the paper fixes it at
                               1 kg/m^3 and optimises the wind (Sec. 3.4).  0 = none  */
  int32_t cg_warm_start;    /* 0: every CG solve starts from 0 (the plain method); 1: each
                               forward solve starts from the previous step's dv and each
                               adjoint solve from the lambda of the step after it (the first
                               solve of a call from 0); the stopping test stays
                               |r| <= cg_tol |b|, so results differ from the zero start by
                               at most what the tolerance allows.  Checkpoint-and-recompute
                               replays the same starting vectors (bitwise the same results) */
} cloth_opts;

#define CLOTH_FORCES_FORCE 0
#define CLOTH_FORCES_VELOCITY 1

#define CLOTH_PRECOND_JACOBI 0
#define CLOTH_PRECOND_BLOCK_JACOBI 1

/* Fill `opts` with defaults: FP32, 1 step, dt 1/30, tol 1e-6, 2000 iterations,
 * no checkpointing, gravity (0, 0, -9.8), clamp_eta 1e-3, GRAPH execution, poll 16,
 * block-Jacobi preconditioner, autotuned CG schedule, forces as forces, no air drag,
 * CG from a zero start. */
void cloth_default_opts(cloth_opts* opts);

typedef struct cloth_mesh cloth_mesh;
typedef struct cloth_batch cloth_batch;

/* Create a sheet from its rest (template) mesh S_1 (Sec. 3.1, "fixed topology").
 * rest_xyz: host [n][3] double, rest positions [m]; tris: host [m][3] int32,
 * consistently wound triangles; pinned: host [n] uint8 (nonzero = pinned) or NULL.
 * Errors: INVALID_ARG (n < 3, m < 1, index out of range), DEGENERATE (zero-area
 * rest triangle), NONMANIFOLD (edge shared by > 2 triangles or opposite winding). */
int cloth_mesh_create(const double* rest_xyz, int32_t n, const int32_t* tris, int32_t m,
                      const uint8_t* pinned, cloth_mesh** out);
int cloth_mesh_destroy(cloth_mesh* mesh);
/* Vertex, triangle and interior-edge (hinge) counts. */
int cloth_mesh_info(const cloth_mesh* mesh, int32_t* n, int32_t* m, int32_t* hinges);

/* Create a batch of `count` sheets sharing `opts` and allocate its device
 * workspace on the current CUDA device (the meshes are copied; they may be
 * destroyed afterwards).  Sheets may differ in size and material. */
int cloth_batch_create(const cloth_mesh* const* meshes, int32_t count, const cloth_opts* opts,
                       cloth_batch** out);
int cloth_batch_destroy(cloth_batch* batch);
/* total_vertices = N_total; workspace_bytes = device memory owned by the handle. */
int cloth_batch_info(const cloth_batch* batch, int32_t* total_vertices, int32_t* count,
                     size_t* workspace_bytes);

/* Forward trajectory (Eq. 1, Eq. 3-5), all sheets at once.
 * material: device [count][4] = (Y [N/m], nu, k_b [N m], rho [kg/m^2]) per sheet;
 * x0, v0: device [N_total][3]; forces: device [steps][N_total][3] newtons (or m/s
 * velocity increments under CLOTH_FORCES_VELOCITY, see cloth_opts.force_mode), or
 * NULL for none; traj_x: device [steps + 1][N_total][3], written (traj_x[0] = x0);
 * status: device [count] int32, written with CLOTH_STATUS_* bits.
 * Keeps internally what cloth_backward needs: a copy of `material` and the
 * checkpointed states.  `forces` is read again by the backward's recompute, so its
 * contents must stay unchanged until the matching cloth_backward has been issued.
 * The state (x, v) is carried in double internally in both precisions; element
 * edge vectors are formed from it before rounding to the batch precision. */
int cloth_forward(cloth_batch* batch, const void* material, const void* x0, const void* v0,
                  const void* forces, void* traj_x, int32_t* status, void* stream);

/* Adjoint of the last cloth_forward on this handle (same inputs assumed).
 * dL_dx: device [steps + 1][N_total][3], gradient of the loss w.r.t. every x_t.
 * Outputs (each may be NULL): g_material [count][4] (dL/dY, 0 for nu, dL/dk_b,
 * dL/drho), g_forces [steps][N_total][3], g_x0 [N_total][3], g_v0 [N_total][3].
 * status as in cloth_forward (adjoint solves).  Error STATE if no forward ran. */
int cloth_backward(cloth_batch* batch, const void* dL_dx, void* g_material, void* g_forces,
                   void* g_x0, void* g_v0, int32_t* status, void* stream);

/* Trajectory loss L_s = sum_{t=1..steps} sum_{i in s} |x_t^i - target_t^i|^2 per
 * sheet (a 3-D surrogate of the image energy of Eq. 7-8, accumulated in double).
 * traj_x, target: device [steps + 1][N_total][3]; loss: device [count] double;
 * dL_dx: device [steps + 1][N_total][3] or NULL (row t = 0 is written as 0). */
int cloth_loss_l2(cloth_batch* batch, const void* traj_x, const void* target, double* loss,
                  void* dL_dx, void* stream);

/* Pinhole reprojection loss per sheet, sum_{t>=1} sum_i |pi(x_t^i) - uv_t^i|^2,
 * with camera (host double[4]) = (f [px], cx, cy, cz): camera centre c looking
 * along -z, pi(x) = f ((x - cx) / (cz - z), -(y - cy) / (cz - z)).
 * target_uv: device [steps + 1][N_total][2]; loss, dL_dx as in cloth_loss_l2.
 * A point with cz - z <= 0 makes its sheet's loss NaN. */
int cloth_loss_pinhole(cloth_batch* batch, const void* traj_x, const void* target_uv,
                       const double* camera, double* loss, void* dL_dx, void* stream);

/* CG iteration totals of the last forward and backward (summed over sheets and
 * steps; the backward's recomputed forward solves are counted apart), and the
 * number of kernels the last forward plus backward launched, CG loop bodies
 * included.  Synchronises the stream of the last call.  Any pointer may be NULL. */
int cloth_stats(cloth_batch* batch, int64_t* fwd_cg_iters, int64_t* bwd_cg_iters,
                int64_t* recompute_cg_iters, int64_t* kernel_launches);

/* Per-sheet CG iteration counts of the last call of one phase: 0 = the solves of
 * cloth_forward, 1 = the adjoint solves of cloth_backward, 2 = the forward solves
 * cloth_backward recomputed from checkpoints, 3 = the solves cloth_time_kernel(5) timed
 * (cleared again when it returns: always 0 here).  max_iters (host [count]): the most
 * iterations one solve of that sheet took; total_iters (host [count]): the sum over
 * its solves.  Either may be NULL.  Synchronises the stream of the last call.
 * Error INVALID_ARG for another phase. */
int cloth_sheet_iterations(cloth_batch* batch, int32_t phase, int32_t* max_iters, int64_t* total_iters);

/* Size of the step matrix A (Eq. 4-5) in 3x3 blocks: rows (vertices, each sheet
 * padded to a multiple of 32), blocks (structurally nonzero blocks) and
 * stored_blocks (blocks stored by the SELL-32 layout, padding included); cg_schedule:
 * the CG kernel schedule in use (0..31, see cloth_opts).  Any pointer may be NULL. */
int cloth_matrix_info(const cloth_batch* batch, int64_t* rows, int64_t* blocks,
                      int64_t* stored_blocks, int32_t* cg_schedule);

/* Average device time [ms] of `reps` back-to-back launches of one step kernel on
 * the state left by the last call, timed with CUDA events on `stream`:
 * kernel 0 = CG SpMV with its per-sheet p^T A p reduction, 1 = CG vector update,
 * 2 = assembly, 3 = membrane element kernel, 4 = bending element kernel, 5 = a whole CG
 * solve (every sheet to convergence, the schedule in use, from zero) of the system the
 * last call assembled last, replayed from one captured graph.  Needs a prior
 * cloth_forward; synchronises `stream`; leaves the solver's scratch (not the handle's
 * saved states) overwritten. */
int cloth_time_kernel(cloth_batch* batch, int32_t kernel, int32_t reps, double* avg_ms,
                      void* stream);

/* Algorithmic bytes of one launch of the kernel cloth_time_kernel times under the same
 * id (compulsory traffic: every input the kernel needs and every output it writes,
 * once; vertex state read once per vertex), for the roofline of that kernel: the SpMV
 * counts the nonzero blocks (9 values + column each) and its vector traffic for the
 * schedule in use; kernel 5 counts, for every sheet, its iterations in the last solve
 * timed as kernel 5 times what kernels 0 and 1 move for its rows (the matrix once per
 * iteration).  No device work; error INVALID_ARG for another id, or for kernel 5 before
 * it was timed. */
int cloth_kernel_bytes(cloth_batch* batch, int32_t kernel, int64_t* bytes);

/* Wind velocity per sheet for the air drag (cloth_opts.air_density > 0): device
 * [count][3] in the batch precision [m/s], or NULL for still air.  The pointer is kept
 * and read by every later cloth_forward and cloth_backward (recompute and adjoint), so
 * its contents must stay unchanged until the matching cloth_backward has been issued;
 * no device work. */
int cloth_set_wind(cloth_batch* batch, const void* wind);

/* dL/dw of the last cloth_backward: device [count][3] in the batch precision, written
 * on `stream` (zero without air drag). */
int cloth_wind_gradient(cloth_batch* batch, void* g_wind, void* stream);

/* ---- single-kernel entry points (parity checks of each stage) ---- */

/* Internal elastic forces f = -dE/dx at positions x (device [N_total][3]):
 * f_membrane and f_bending device [N_total][3] (either may be NULL). */
int cloth_internal_forces(cloth_batch* batch, const void* material, const void* x,
                          void* f_membrane, void* f_bending, void* stream);

/* The linear system of one step (Eq. 4-5) at state (x, v) with external force
 * F (device [N_total][3] or NULL; under CLOTH_FORCES_VELOCITY a velocity increment,
 * the step then starting from v + F), assembled by the step kernels and expanded to
 * dense per sheet: A: device [sum_s (3 n_s)^2] (sheet blocks one after another,
 * row-major, user vertex order), b: device [N_total][3].  Pinned rows and
 * columns are identity, b = 0 there.  For small sheets (testing). */
int cloth_system_dense(cloth_batch* batch, const void* material, const void* x, const void* v,
                       const void* F, void* A, void* b, void* stream);

/* y = A p with the assembled system at (x, v) (the CG's SpMV kernel).
 * p, y: device [N_total][3]. */
int cloth_spmv(cloth_batch* batch, const void* material, const void* x, const void* v,
               const void* p, void* y, void* stream);

/* D^3E(x)[a, b, .] for the matrix Hessian (clamped membrane + bending), the
 * third-derivative contraction of the adjoint: out device [N_total][3]. */
int cloth_third_contraction(cloth_batch* batch, const void* material, const void* x,
                            const void* a, const void* b, void* out, void* stream);

/* ---- image energies of a sheet (Sec. 3.2) ----
 *
 * Soft rasterisation of one textured sheet and its photometric and silhouette energies,
 * E = E_p + lambda E_s, E_p = sum_pixels |I - I_hat|_1 (RGB), E_s = sum_pixels
 * |G(A) - G(B_hat)|_1 with G the Gaussian filter of 7 px (lambda = 0.5), and dE/dx.
 * The rasteriser: coverage sigmoid(+-d^2 / 1 px^2) of each projected triangle (d: distance
 * of the pixel centre to its nearest edge, + inside), silhouette A = 1 - prod(1 - D),
 * bilinear texture colour at the clamped barycentric uv, blended against a black
 * background with weights D exp(zn / 1e-4) (zn: normalised inverse depth, 1 at 0.5 m,
 * 0 at 5 m; background zn 1e-3).  Camera: the pinhole of cloth_loss_pinhole with the
 * principal point at the image centre, pixel centres at (u + 1/2, v + 1/2).
 * n vertices, m triangles: tris HOST [m][3] (validated: INVALID_ARG if out of range);
 * x device [n][3], uv device [n][2] (texture coordinates in [0, 1]^2, v down the
 * texture), tex device [tex_h][tex_w][3], camera HOST double[4] (f, cx, cy, cz);
 * image device [H][W][3], mask device [H][W] (the input frame and its foreground mask);
 * scratch: device, cloth_image_energy_scratch(n, m, W, H) bytes, 8-byte aligned;
 * energy: device double[1]; dE_dx: device [n][3] or NULL; out_image [H][W][3] and
 * out_silhouette [H][W]: device or NULL.  All arrays double; all work on `stream`. */
size_t cloth_image_energy_scratch(int32_t n, int32_t m, int32_t W, int32_t H);
int cloth_image_energy(int32_t n, int32_t m, const int32_t* tris, const double* x, const double* uv,
                       int32_t tex_w, int32_t tex_h, const double* tex, const double* camera, int32_t W,
                       int32_t H, const double* image, const double* mask, void* scratch, double* energy,
                       double* dE_dx, double* out_image, double* out_silhouette, void* stream);

/* ---- allocation-free variant (the paper has no counterpart) ----
 *
 * cloth_loss_l2_static computes exactly what cloth_loss_l2 computes (same kernels,
 * per-sheet loss sum_{t=1..steps} sum_i |x_t^i - target_t^i|^2 in double and, when
 * dL_dx is non-NULL, its gradient with row t = 0 set to 0) but needs no batch handle and
 * never allocates device memory.  It is meant for callers that must not call
 * cudaMalloc at the point of use: code running where another allocator owns the device
 * memory (a framework that has reserved the whole pool), or latency-critical loops where
 * the implicit device synchronisation of cudaMalloc/cudaFree would stall the pipeline.
 * Its scratch (one double per sheet and time step) is a static array of 65,536 doubles
 * (512 KiB) that every GPU loading this library holds until the process exits; calls
 * with count * steps > 65,536 (or count or steps > 65,535) fail with
 * CLOTH_ERR_INVALID_ARG.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current and keeps it for the life of
 * the process; make that first call before any stream capture, and do not call this entry
 * point on a device after a cudaDeviceReset of it (the kept address is then stale).
 * Devices with an index of 64 or more are rejected with CLOTH_ERR_INVALID_ARG.  All calls share the one array: calls whose kernels overlap on the
 * GPU (e.g. issued to different streams without ordering) race and give wrong losses.
 * count: sheets; sheet_offsets: device [count + 1] int32, vertex offset of each sheet in
 * the packed user layout (sheet_offsets[count] = n_total); steps, n_total: as in
 * cloth_loss_l2; precision: CLOTH_FP32 or CLOTH_FP64 (type of traj_x, target, dL_dx);
 * traj_x, target: device [steps + 1][n_total][3]; loss: device [count] double;
 * dL_dx: device [steps + 1][n_total][3] or NULL. */
int cloth_loss_l2_static(int32_t count, const int32_t* sheet_offsets, int32_t steps, int32_t n_total,
                         int32_t precision, const void* traj_x, const void* target, double* loss,
                         void* dL_dx, void* stream);

/* Thread-local description of the last error (empty string if none). */
const char* cloth_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CLOTH_SIM_H */
