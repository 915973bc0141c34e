"""Adam driver with the adaptive temporal window of phi-SfT (Sec. 3.3 "Adaptive
Optimisation Scheme", Sec. 3.4 implementation details) over a synthetic pinhole-track
loss: recovers the material (Y, k_b, rho) and the per-step corrective forces of one or
more sheets from 2-D tracks.

Every forward, loss and adjoint runs in the CUDA library (`sim.ClothBatch`); this module
holds only the host-side schedule and the optimiser update (torch.optim.Adam on device
tensors).  Readings of the paper:

* Window: the first 5 frames are active at the start.  The threshold b is defined as the
  energy frame 5 has when frame 6 is added, so the first extension happens when the
  per-window iteration cap is reached; afterwards the next frame is added as soon as the
  latest active frame's energy drops below b, or when the cap is reached.
* The energy of frame t is the pinhole reprojection energy sum_i |pi(x_t^i) - u_t^i|^2
  of tracked points, or (image_frame_loss) the paper's image energy E_p + 0.5 E_s of the
  soft-rasterised sheet against the input frame and its mask.  The simulation runs the full
  trajectory every iteration; frames after the active one get zero loss gradient, which
  gives the same gradient as simulating only the active frames.
* Adam with learning rate 1e-3 on log Y, log k_b, log rho (the parameters span decades)
  and on the corrective forces directly; nu is not optimised.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class AdaptiveWindow:
    """Host-side state of the adaptive temporal window (frames are 1..T; frame 0 is the
    given initial state)."""

    total: int                 # T, the number of frames after the initial state
    first: int = 5             # frames active at the start
    max_iters: int = 50        # iterations after which the window grows regardless
    active: int = field(init=False)
    threshold: float = field(init=False, default=float("inf"))
    iters: int = field(init=False, default=0)

    def __post_init__(self):
        self.active = min(self.first, self.total)

    @property
    def done(self):
        return self.active >= self.total

    def step(self, frame_energy):
        """Account one optimisation iteration with the per-frame energies
        frame_energy[t] (t = 0..T) measured in it; returns True when a frame was added."""
        self.iters += 1
        if self.done:
            return False
        first_growth = not np.isfinite(self.threshold)
        reached = (not first_growth) and frame_energy[self.active] < self.threshold
        if reached or self.iters >= self.max_iters:
            if first_growth:
                self.threshold = float(frame_energy[min(self.first, self.total)])
            self.active += 1
            self.iters = 0
            return True
        return False


def project(traj, camera):
    """Pinhole projection of every vertex of a trajectory [T+1, N, 3] (the convention of
    cloth_loss_pinhole: centre (cx, cy, cz) looking along -z, image axes (x, -y))."""
    import torch

    f, cx, cy, cz = camera
    depth = cz - traj[..., 2]
    return torch.stack([f * (traj[..., 0] - cx) / depth, -f * (traj[..., 1] - cy) / depth], dim=-1)


def frame_energies(traj, tracks, camera):
    """Per-frame reprojection energy sum_i |pi(x_t^i) - u_t^i|^2, [T+1] (summed over sheets)."""
    d = project(traj.double(), camera) - tracks.double()
    return (d * d).sum(dim=(1, 2))


def image_frame_loss(images, masks, tris, uv, tex, camera, energy_fn=None):
    """Per-frame loss of a one-sheet batch against input frames: the image energy
    E_p + 0.5 E_s of each frame t >= 1 (cloth_image_energy).  images[t] [H, W, 3] and
    masks[t] [H, W] (CUDA float64), tris [m, 3] (host), uv [n, 2], tex [Ht, Wt, 3].
    energy_fn(x_t, t) -> (E, dE/dx_t) replaces the library call (tests).  Returns
    loss(traj) -> (per-frame energies [T+1], dL/dx [T+1, n, 3])."""

    def gpu_energy(xt, t):
        from . import sim

        E, g, _, _ = sim.image_energy(xt, tris, uv, tex, camera, images[t], masks[t])
        return E[0], g

    fn = energy_fn or gpu_energy

    def loss(traj):
        import torch

        e = torch.zeros(traj.shape[0], dtype=torch.float64)
        dL = torch.zeros_like(traj)
        for t in range(1, traj.shape[0]):
            E, g = fn(traj[t].double().contiguous(), t)
            e[t] = float(E)
            dL[t] = g.to(traj.dtype)
        return e, dL

    return loss


@dataclass
class FitResult:
    material: np.ndarray       # [S, 4]
    forces: np.ndarray         # [T, N, 3]
    history: list              # per iteration: (active frames, energy of the active frames)
    window: AdaptiveWindow
    materials: list = field(default_factory=list)  # per iteration: the material [S, 4] it simulated


def fit(batch, material0, x0, v0, tracks, camera, *, forces0=None, iters=200, lr=1e-3, first=5, max_iters=50,
        optimise_forces=True, frame_loss=None):
    """Adam over (log Y, log k_b, log rho) of every sheet and the per-step forces, with
    the adaptive window.  batch: a sim.ClothBatch; material0 [S, 4], x0/v0 [N, 3],
    tracks [T+1, N, 2] (device tensors of the batch's precision) for the pinhole-track
    loss, or frame_loss(traj) -> (per-frame energies [T+1], dL/dx [T+1, N, 3]) in its
    place (e.g. image_frame_loss; tracks and camera are then unused).  batch may be any
    object with the same steps, forward, loss_pinhole and backward (the tests drive the
    same schedule through the oracle that way)."""
    import torch

    dtype = x0.dtype
    T = batch.steps
    logm = torch.log(material0[:, [0, 2, 3]].clone().double()).requires_grad_(True)
    nu = material0[:, 1].clone()
    F = (forces0.clone() if forces0 is not None else
         torch.zeros(T, x0.shape[0], 3, dtype=dtype, device=x0.device)).double().requires_grad_(optimise_forces)
    params = [logm] + ([F] if optimise_forces else [])
    opt = torch.optim.Adam(params, lr=lr)
    window = AdaptiveWindow(T, first=first, max_iters=max_iters)
    history, materials = [], []
    # fixed input buffers: the library caches one captured graph per set of argument addresses
    mat = torch.empty(material0.shape, dtype=dtype, device=x0.device)
    Fc = torch.empty(T, x0.shape[0], 3, dtype=dtype, device=x0.device)
    for _ in range(iters):
        m = torch.exp(logm.detach())
        mat.copy_(torch.stack([m[:, 0], nu.double(), m[:, 1], m[:, 2]], dim=1))
        Fc.copy_(F.detach())
        traj, status = batch.forward(mat, x0, v0, Fc)
        if frame_loss is None:
            _, dL = batch.loss_pinhole(traj, tracks, camera)
            e = frame_energies(traj, tracks, camera)
        else:
            e, dL = frame_loss(traj)
        dL[window.active + 1:] = 0  # frames after the active one do not take part
        g = batch.backward(dL)
        history.append((window.active, float(e[1:window.active + 1].sum())))
        materials.append(mat.detach().double().cpu().numpy().copy())
        opt.zero_grad()
        gm = g["material"].double()
        logm.grad = torch.stack([gm[:, 0], gm[:, 2], gm[:, 3]], dim=1) * m  # chain rule through exp
        if optimise_forces:
            F.grad = g["forces"].double()
        opt.step()
        window.step(np.asarray(e.detach().cpu() if hasattr(e, "cpu") else e, dtype=np.float64))
    m = torch.exp(logm.detach())
    mat = torch.stack([m[:, 0], nu.double(), m[:, 1], m[:, 2]], dim=1)
    return FitResult(mat.cpu().numpy(), F.detach().cpu().numpy(), history, window, materials)
