"""Learned closure for a 2x-coarsened acoustic-wave solve: wrapper and training driver.

The network, its backward pass and Adam run in ``libgbstencil.so``
(``closure_*`` entry points); the fine and coarse solves are the library's
stencil sweeps.  This module only orchestrates: it builds the fine (h) and
coarse (2h, 2 dt) grids of one seeded layered model, restricts the fine
solution onto the coarse grid by injection (every second point, the library's
strided read), trains the closure on one-step corrections, and evaluates
plain and corrected coarse runs against the restricted fine solution.

Inputs: s (u+, u^n, c_n^2 u+, c_n^2 u^n) with c_n = c / 4500 -- every channel
vanishes with the field, so with zero, frozen biases a zero field receives an
exactly zero correction (a constant velocity channel made rollouts diverge).

Reading of the set-up (the paper has no learned part): the point source is
volume-normalised, so the coarse grid injects (h_f / h_c)^3 = 1/8 of the fine
amplitude per unit of c^2 dt^2 R(t); with dt_c = 2 dt_f the CFL number of both
grids is the same.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import native as N
from .grid import Grid, TorchAllocator

C_REF = 4500.0


class Closure:
    """One closure network (``closure_create``) with torch-owned device memory."""

    def __init__(self, max_points: int, in_scale: float, cin: int = 4, hidden: int = 16, stream=None,
                 torch_allocator: bool = True):
        import torch
        self._torch = torch
        dev = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self._alloc = TorchAllocator(dev) if torch_allocator else None
        self.h = N.closure_create(cin, hidden, max_points, in_scale, self.stream.cuda_stream,
                                  self._alloc.struct if self._alloc else None)
        self.nparams = N.closure_param_count(self.h)
        self.scale = in_scale
        self.out_scale = in_scale

    def set_params(self, flat: np.ndarray):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.nparams
        N.closure_set_params(self.h, a.ctypes.data, a.size)

    def get_params(self) -> np.ndarray:
        out = np.empty(self.nparams, dtype=np.float32)
        N.closure_get_params(self.h, out.ctypes.data, out.size)
        return out

    def get_grads(self) -> np.ndarray:
        out = np.empty(self.nparams, dtype=np.float32)
        N.closure_get_grads(self.h, out.ctypes.data, out.size)
        return out

    def _sync_in(self):
        self.stream.wait_stream(self._torch.cuda.current_stream())

    def forward(self, up, un, cn):
        """Correction o / s for dense (nz, ny, nx) FP32 CUDA tensors."""
        self._sync_in()
        out = self._torch.empty_like(up)
        dims = tuple(reversed(up.shape))
        N.closure_forward(self.h, up.data_ptr(), un.data_ptr(), cn.data_ptr(), dims, out.data_ptr())
        self._torch.cuda.current_stream().wait_stream(self.stream)
        return out

    def loss_grad(self, up, un, cn, ref) -> float:
        self._sync_in()
        dims = tuple(reversed(up.shape))
        return N.closure_loss_grad(self.h, up.data_ptr(), un.data_ptr(), cn.data_ptr(), ref.data_ptr(), dims)

    def adam_step(self, lr: float):
        N.closure_adam_step(self.h, lr)

    def set_out_scale(self, v: float):
        N.closure_set_out_scale(self.h, v)
        self.out_scale = v

    def set_loss_weight(self, w: float):
        N.closure_set_loss_weight(self.h, w)

    def freeze_biases(self, on: bool = True):
        N.closure_freeze_biases(self.h, on)

    def set_features(self, space_order: int, scales):
        """Feature inputs (closures created with cin = 8): channel scales and the star's order."""
        N.closure_set_features(self.h, space_order, scales)
        self.feature_scales = list(scales)

    def feature_values(self, up, un, cn):
        """The eight unscaled FP32 features, shape (8, nz, ny, nx)."""
        self._sync_in()
        out = self._torch.empty((8,) + tuple(up.shape), dtype=self._torch.float32, device=up.device)
        N.closure_feature_values(self.h, up.data_ptr(), un.data_ptr(), cn.data_ptr(), tuple(reversed(up.shape)),
                                 out.data_ptr())
        self._torch.cuda.current_stream().wait_stream(self.stream)
        return out

    def set_conv_impl(self, impl: int):
        """0: tcgen05 convolutions (default); 1: mma.sync convolutions; 2: tcgen05 for the
        hidden layers, the one-channel last layer on the CUDA cores."""
        N.closure_set_conv_impl(self.h, impl)

    def close(self):
        if getattr(self, "h", None):
            N.closure_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def flatten_params(p: dict) -> np.ndarray:
    """Oracle-order flat vector w1, b1, w2, b2, w3, b3."""
    return np.concatenate([np.asarray(p[k], dtype=np.float32).reshape(-1)
                           for k in ("w1", "b1", "w2", "b2", "w3", "b3")])


def unflatten_params(flat: np.ndarray, cin: int = 4, hidden: int = 16) -> dict:
    shapes = [("w1", (hidden, cin, 3, 3, 3)), ("b1", (hidden,)), ("w2", (hidden, hidden, 3, 3, 3)),
              ("b2", (hidden,)), ("w3", (1, hidden, 3, 3, 3)), ("b3", (1,))]
    out, o = {}, 0
    for k, shp in shapes:
        n = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


# ----------------------------------------------------------------- set-up ---

@dataclasses.dataclass
class PairConfig:
    nc: int = 256          # coarse points per axis (fine: 2 nc)
    hf: float = 10.0       # fine spacing (m); coarse 2 hf
    so: int = 4
    f0: float = 10.0
    steps: int = 400       # coarse steps
    cfl_frac: float = 0.5  # of the stability limit


def _courant_max(ndim: int, so: int) -> float:
    import synthetic
    return synthetic.wave_courant_max(ndim, so)


class FineCoarsePair:
    """Fine (2 nc)^3 grid with spacing hf and coarse nc^3 grid with 2 hf of one seeded model."""

    def __init__(self, seed: int, cfg: PairConfig, stream=None):
        import torch
        import synthetic
        self.torch = torch
        self.cfg = cfg
        self.stream = stream if stream is not None else torch.cuda.Stream()
        nc, nf = cfg.nc, 2 * cfg.nc
        self.nc, self.nf = nc, nf
        speeds = synthetic.seeded_layer_speeds(seed)
        self.cf = synthetic.layered_velocity((nf, nf, nf), speeds)
        self.cc = np.ascontiguousarray(self.cf[::2, ::2, ::2])
        self.dtf = cfg.cfl_frac * _courant_max(3, cfg.so) * cfg.hf / max(speeds)
        self.dtc = 2.0 * self.dtf
        # source near the middle of the coarse grid, on a point shared with the fine grid
        u = synthetic.uniform01(seed, 3, start=500).astype(np.float64)
        self.src_c = tuple(int(nc // 2 - nc // 8 + np.floor(v * (nc // 4))) for v in u)
        self.src_f = tuple(2 * s for s in self.src_c)
        self.fine = Grid(3, (nf,) * 3, cfg.so, "wave", h=cfg.hf, dt=self.dtf, stream=self.stream)
        self.fine.set_field("vel", self.cf)
        self.fine.set_source(self.src_f, cfg.f0, 1.0 / cfg.f0, 1.0)
        self.coarse = Grid(3, (nc,) * 3, cfg.so, "wave", h=2 * cfg.hf, dt=self.dtc, stream=self.stream)
        self.coarse.set_field("vel", self.cc)
        self.coarse.set_source(self.src_c, cfg.f0, 1.0 / cfg.f0, 1.0 / 8.0)
        cn = (self.cc / C_REF).astype(np.float32)
        self.cnorm = torch.from_numpy(cn).cuda()

    def restrict(self, out=None):
        """Fine u at even indices (injection), as a dense (nc, nc, nc) FP32 CUDA tensor."""
        t = self.torch
        if out is None:
            out = t.empty((self.nc,) * 3, dtype=t.float32, device="cuda")
        N.stencil_get_field_strided(self.fine.h, N.GBST_U, out.data_ptr(), 2)
        return out

    def close(self):
        self.fine.close()
        self.coarse.close()


def coarse_step(pair: FineCoarsePair, u_cur, u_prev, n: int, out):
    """One plain coarse step from (u^n, u^{n-1}) at step index n; u^{n+1} into `out`."""
    g = pair.coarse
    g.set_field("u", u_cur)
    g.set_field("u_prev", u_prev)
    g.step = n
    g.run(1)
    g.get_field("u", out=out)
    return out


def field_scale(seed: int, cfg: PairConfig) -> float:
    """1 / max |u| of the restricted fine solution over a trajectory (sampled every 8 coarse steps)."""
    import torch
    pair = FineCoarsePair(seed, cfg)
    m = 0.0
    r = torch.empty((pair.nc,) * 3, dtype=torch.float32, device="cuda")
    for n in range(0, cfg.steps, 8):
        pair.fine.run(16)
        m = max(m, float(pair.restrict(r).abs().max()))
    pair.close()
    return 1.0 / m if m > 0 else 1.0


def zero_last_layer(flat: np.ndarray, cin: int = 4, hidden: int = 16) -> np.ndarray:
    """Parameters with w3 = b3 = 0: the closure starts as 'no correction'."""
    out = np.array(flat, dtype=np.float32, copy=True)
    n3 = hidden * 27 + 1
    out[-n3:] = 0.0
    return out


def zero_biases(flat: np.ndarray, cin: int = 4, hidden: int = 16) -> np.ndarray:
    p = unflatten_params(flat, cin, hidden)
    for k in ("b1", "b2", "b3"):
        p[k][...] = 0.0
    return flatten_params(p)


def correction_scale(seed: int, cfg: PairConfig, quantile: float = 0.999, n_start: int = 0) -> float:
    """1 / (the `quantile` of the per-step max |u_ref - u+|) over steps >= n_start of one trajectory."""
    import torch
    pair = FineCoarsePair(seed, cfg)
    shp = (pair.nc,) * 3
    r_prev = torch.zeros(shp, dtype=torch.float32, device="cuda")
    r_cur = torch.zeros(shp, dtype=torch.float32, device="cuda")
    r_next = torch.empty(shp, dtype=torch.float32, device="cuda")
    up = torch.empty(shp, dtype=torch.float32, device="cuda")
    vals = []
    for n in range(cfg.steps):
        coarse_step(pair, r_cur, r_prev, n, up)
        pair.fine.run(2)
        pair.restrict(r_next)
        if n % 4 == 0 and n >= n_start:
            d = (r_next - up).abs().flatten()
            vals.append(float(d.max()))
        r_prev, r_cur, r_next = r_cur, r_next, r_prev
    pair.close()
    m = float(np.quantile(np.asarray(vals), quantile)) if vals else 1.0
    return 1.0 / m if m > 0 else 1.0


def train(closure: Closure, seeds, cfg: PairConfig, lr: float = 2e-3, epochs: int = 1, lr_final: float = None,
          crop: int = 0, updates_per_step: int = 1, seed: int = 0, normalise: bool = False, n_start: int = 1,
          log=None):
    """Train on one-step corrections along fine trajectories (teacher forcing).

    Updates use coarse steps n >= max(1, n_start) (the trajectory before is
    replayed without updates).
    Every epoch replays each seed's fine trajectory (cheap next to the network,
    so no samples are stored); at each coarse step the plain coarse step from the
    restricted fine state is compared with the restricted next fine state.  With
    crop > 0 each update uses a random crop^3 window of the coarse grid (the
    closure is local, so windows are enough and keep updates cheap).  The
    learning rate decays geometrically from lr to lr_final (default lr / 20).
    """
    import torch
    losses = []
    t0 = time.time()
    n_start = max(1, n_start)
    total = max(1, epochs * len(seeds) * (cfg.steps - n_start) * updates_per_step)
    lr_final = lr / 20 if lr_final is None else lr_final
    rng = np.random.default_rng(seed)
    k = 0
    for ep in range(epochs):
        for sd in seeds:
            pair = FineCoarsePair(sd, cfg)
            shp = (pair.nc,) * 3
            r_prev = torch.zeros(shp, dtype=torch.float32, device="cuda")
            r_cur = torch.zeros(shp, dtype=torch.float32, device="cuda")
            r_next = torch.empty(shp, dtype=torch.float32, device="cuda")
            up = torch.empty(shp, dtype=torch.float32, device="cuda")
            w = crop if 0 < crop < pair.nc else pair.nc
            for n in range(cfg.steps):
                coarse_step(pair, r_cur, r_prev, n, up)
                pair.fine.run(2)
                pair.restrict(r_next)
                if n >= n_start:
                    for _ in range(updates_per_step):
                        if w < pair.nc:
                            o = rng.integers(0, pair.nc - w + 1, size=3)
                            sl = (slice(o[0], o[0] + w), slice(o[1], o[1] + w), slice(o[2], o[2] + w))
                            args = [t[sl].contiguous() for t in (up, r_cur, pair.cnorm, r_next)]
                        else:
                            args = [up, r_cur, pair.cnorm, r_next]
                        if normalise:
                            ms = float(((args[3] - args[0]) ** 2).mean()) * closure.out_scale ** 2
                            if ms <= 0:
                                continue
                            closure.set_loss_weight(1.0 / ms)
                        losses.append(closure.loss_grad(*args))
                        closure.adam_step(lr * (lr_final / lr) ** (k / total))
                        k += 1
                r_prev, r_cur, r_next = r_cur, r_next, r_prev
            pair.close()
            if log:
                log(f"epoch {ep} seed {sd}: {len(losses)} updates, mean loss of the last 50 "
                    f"{np.mean(losses[-50:]) if losses else float('nan'):.3e}, {time.time() - t0:.1f}s")
    return losses


def init_params(cin: int = 4, hidden: int = 16, seed: int = 5) -> np.ndarray:
    """Seeded uniform initial weights (bound 1 / sqrt(fan_in)), zero biases, zero last layer."""
    import synthetic
    shapes = [(hidden, cin, 3, 3, 3), (hidden,), (hidden, hidden, 3, 3, 3), (hidden,), (1, hidden, 3, 3, 3), (1,)]
    parts, off = [], 0
    for li, shp in enumerate(shapes):
        n = int(np.prod(shp))
        if li in (1, 3, 4, 5):
            parts.append(np.zeros(n, dtype=np.float32))
        else:
            fan_in = (cin if li == 0 else hidden) * 27
            u = synthetic.uniform01(seed, n, start=off).astype(np.float64)
            parts.append(((2.0 * u - 1.0) / np.sqrt(fan_in)).astype(np.float32))
        off += n
    return np.concatenate(parts)


def new_closure(cfg: PairConfig, max_points: int, scale_seed: int = 10, init_seed: int = 5,
                stream=None, n_start: int = 0) -> Closure:
    """A closure with data-derived input/output scales, zero last layer and zero, frozen biases.

    The output scale comes from the one-step corrections of steps >= n_start."""
    s = field_scale(scale_seed, cfg)
    t = correction_scale(scale_seed, cfg, n_start=n_start)
    cl = Closure(max_points, s, stream=stream)
    cl.set_out_scale(t)
    cl.freeze_biases(True)
    cl.set_params(init_params(seed=init_seed))
    return cl


def rel_l2(a, b) -> float:
    return float((a - b).norm() / b.norm())


def evaluate(closure: Closure, seed: int, cfg: PairConfig, checkpoints=None, attach_at: int = 0,
             detach_at: int | None = None, guard: float | None = 2.0, guard_every: int = 25):
    """Plain coarse, closure-corrected coarse and restricted fine solutions.

    Returns the relative L2 errors (vs the restricted fine solution) at the
    last step, the gain err_plain / err_closure, wall times of the three solves,
    and the errors at the intermediate checkpoints.  The closure corrects steps
    attach_at <= n < detach_at (outside that window the corrected run takes plain
    coarse steps).

    Guard (the plain coarse solve as the fallback and judge of the corrected one):
    every guard_every steps the FP64 L2 norms of the two coarse fields are
    compared (stencil_reduce_f64); if the corrected field's norm exceeds the plain
    one's by more than the relative bound `guard` (or is not finite), the closure
    is detached and the corrected grid continues from the plain grid's levels, i.e.
    as the plain solve.  It is a divergence detector: an unstable correction grows
    without bound and trips any bound within a few checks, while a good correction
    may legitimately move the norm far from the plain coarse one in the source phase
    (the 4-channel network at 96^3 raises it by 57 % at step 25 while cutting the
    error from 52 % to 16 %); hence the default of 2 (three times the plain norm).
    guard=None disables it.
    """
    import torch
    extra = ([attach_at] if attach_at > 0 else []) + ([detach_at] if detach_at else [])
    checkpoints = sorted(set(list(checkpoints or []) + [cfg.steps] + extra))
    pair = FineCoarsePair(seed, cfg)
    shp = (pair.nc,) * 3
    g = Grid(3, shp, cfg.so, "wave", h=2 * cfg.hf, dt=pair.dtc, stream=closure.stream)
    g.set_field("vel", pair.cc)
    g.set_source(pair.src_c, cfg.f0, 1.0 / cfg.f0, 1.0 / 8.0)
    attached = attach_at <= 0
    if attached:
        N.stencil_attach_closure(g.h, closure.h, C_REF)
    ref = torch.empty(shp, dtype=torch.float32, device="cuda")
    u_plain = torch.empty(shp, dtype=torch.float32, device="cuda")
    u_cl = torch.empty(shp, dtype=torch.float32, device="cuda")
    curve = {}
    t_fine = t_plain = t_cl = 0.0
    done = 0
    tripped = None
    worst = 0.0
    for cp in checkpoints:
        while done < cp:
            k = min(cp - done, guard_every) if guard else cp - done
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pair.fine.run(2 * k)
            pair.fine.sync()
            t_fine += time.perf_counter() - t0
            t0 = time.perf_counter()
            pair.coarse.run(k)
            pair.coarse.sync()
            t_plain += time.perf_counter() - t0
            t0 = time.perf_counter()
            g.run(k)
            g.sync()
            t_cl += time.perf_counter() - t0
            done += k
            if guard and attached:
                npl, ncl = pair.coarse.reduce("l2sq"), g.reduce("l2sq")
                dev = (np.sqrt(ncl) - np.sqrt(npl)) / np.sqrt(npl) if npl > 0 else 0.0
                worst = max(worst, dev)
                if not np.isfinite(dev) or dev > guard:
                    N.stencil_attach_closure(g.h, None, C_REF)
                    attached = False
                    tripped = done
                    pair.coarse.get_field("u", out=u_plain)
                    g.set_field("u", u_plain)
                    pair.coarse.get_field("u_prev", out=u_plain)
                    g.set_field("u_prev", u_plain)
        if cp == attach_at and tripped is None:
            N.stencil_attach_closure(g.h, closure.h, C_REF)
            attached = True
        if detach_at and cp == detach_at:
            N.stencil_attach_closure(g.h, None, C_REF)
            attached = False
        pair.restrict(ref)
        pair.coarse.get_field("u", out=u_plain)
        g.get_field("u", out=u_cl)
        curve[cp] = (rel_l2(u_plain, ref), rel_l2(u_cl, ref))
    e_plain, e_cl = curve[cfg.steps]
    out = {"rel_l2_plain_coarse": e_plain, "rel_l2_closure": e_cl, "gain": e_plain / e_cl,
           "seconds_fine": t_fine, "seconds_plain_coarse": t_plain, "seconds_closure": t_cl,
           "steps": cfg.steps, "coarse": pair.nc, "fine": pair.nf, "attach_at": attach_at, "detach_at": detach_at,
           "guard": {"bound": guard, "every": guard_every, "tripped_at": tripped,
                     "largest_norm_excess": worst},
           "curve": {str(k): {"plain": v[0], "closure": v[1]} for k, v in curve.items()}}
    g.close()
    pair.close()
    return out


# ------------------------------------------------- feature inputs, rollouts ---
#
# Reading of the learned part (none of it is in the paper): the network's
# inputs are FP32 stencil features of the coarse field (closure_set_features),
# among them the two leading one-step defects of the order-4 leapfrog scheme,
# kappa sum_a delta_a^6 u / 90 (spatial truncation) and kappa L(kappa L u) / 12
# (the dt^4 u_tttt / 12 term), which BF16 inputs of the raw field cannot resolve
# (they are ~1e-4 of the field and need sixth differences).  The network starts
# as exactly that modified-equation correction (GELU(x) - GELU(-x) = x gives
# linear pass-through channels) and is then trained on coarse-grid rollouts
# against the restricted fine solution, by backpropagation through the time
# steps (stencil_closure_rollout_grad), on windows after the source has died
# out, where the error that remains at the last step is made.

FEATURE_SPACE_ORDER = 4
TAP_CENTRE = 13  # (dz, dy, dx) = (0, 0, 0) in the [3][3][3] tap order


def kappa_ref(pair: "FineCoarsePair") -> float:
    """kappa = kappa_ref * (c / C_REF)^2 on the coarse grid."""
    return (C_REF * pair.dtc / (2.0 * pair.cfg.hf)) ** 2


def feature_scales(seed: int, cfg: PairConfig, every: int = 8) -> list:
    """1 / max |f_k| of the eight features along the restricted fine trajectory of one seed
    (features of consecutive restricted levels; sampled every `every` coarse steps)."""
    import torch
    from . import native as NN
    pair = FineCoarsePair(seed, cfg)
    nc = pair.nc
    cl = Closure(nc ** 3, 1.0, cin=8)
    cl.set_features(FEATURE_SPACE_ORDER, [1.0] * 8)
    shp = (nc,) * 3
    r_prev = torch.zeros(shp, dtype=torch.float32, device="cuda")
    r_cur = torch.zeros_like(r_prev)
    up = torch.empty_like(r_prev)
    m = np.zeros(8)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for n in range(cfg.steps):
        if n % every == 0 and n > 0:
            coarse_step(pair, r_cur, r_prev, n, up)
            f = cl.feature_values(up, r_cur, pair.cnorm)
            torch.cuda.synchronize()
            for k in range(8):
                NN.gbst_reduce_dense_f64_noalloc(f[k].data_ptr(), NN.GBST_F32, f[k].numel(), NN.GBST_RED_MAXABS,
                                                 out.data_ptr(), torch.cuda.current_stream().cuda_stream)
                torch.cuda.synchronize()
                m[k] = max(m[k], float(out.item()))
        pair.fine.run(2)
        nxt = pair.restrict()
        r_prev, r_cur = r_cur, nxt
    cl.close()
    pair.close()
    return [1.0 / v if v > 0 else 1.0 for v in m]


def modified_equation_params(scales, t: float, kref: float, a: float = 1.0, b: float = 1.0, cin: int = 8,
                             hidden: int = 16, seed: int = 5, spread: float = 0.05) -> np.ndarray:
    """Parameters of the network that computes exactly o / t = a kref f4 / 90 + b kref^2 f5 / 12
    through four linear pass-through channels (hidden 0, 1 = +x4, -x4; 2, 3 = +x5, -x5; layer 2
    repeats the differences y(+) - y(-), which equal the inputs since GELU(x) - GELU(-x) = x).
    The other hidden channels start with small seeded weights and no path to the output."""
    import synthetic
    w1 = np.zeros((hidden, cin, 27))
    w2 = np.zeros((hidden, hidden, 27))
    w3 = np.zeros((1, hidden, 27))
    c = TAP_CENTRE
    w1[0, 4, c], w1[1, 4, c], w1[2, 5, c], w1[3, 5, c] = 1.0, -1.0, 1.0, -1.0
    for k, (p_, m_) in enumerate(((0, 1), (2, 3))):
        w2[2 * k, p_, c], w2[2 * k, m_, c] = 1.0, -1.0
        w2[2 * k + 1, p_, c], w2[2 * k + 1, m_, c] = -1.0, 1.0
    alpha = a * t * kref / (90.0 * scales[4])
    beta = b * t * kref * kref / (12.0 * scales[5])
    w3[0, 0, c], w3[0, 1, c], w3[0, 2, c], w3[0, 3, c] = alpha, -alpha, beta, -beta
    # the free channels 4..15: seeded weights within 1/sqrt(fan_in) * spread, no output path yet
    u1 = synthetic.uniform01(seed, (hidden - 4) * cin * 27).astype(np.float64).reshape(hidden - 4, cin, 27)
    w1[4:] = (2 * u1 - 1) * spread / np.sqrt(cin * 27)
    u2 = synthetic.uniform01(seed, (hidden - 4) * hidden * 27, start=10 ** 6).astype(np.float64)
    w2[4:] = ((2 * u2 - 1) * spread / np.sqrt(hidden * 27)).reshape(hidden - 4, hidden, 27)
    p = {"w1": w1.reshape(hidden, cin, 3, 3, 3), "b1": np.zeros(hidden), "w2": w2.reshape(hidden, hidden, 3, 3, 3),
         "b2": np.zeros(hidden), "w3": w3.reshape(1, hidden, 3, 3, 3), "b3": np.zeros(1)}
    return flatten_params(p)


def output_weight_mask(cin: int = 8, hidden: int = 16, channels=(0, 1, 2, 3), taps: str = "centre") -> np.ndarray:
    """Trainable-parameter mask (closure_set_trainable) selecting the last layer's weights from the
    given hidden channels: their centre taps ("centre") or all 27 taps ("all")."""
    n = hidden * cin * 27 + hidden + hidden * hidden * 27 + hidden + hidden * 27 + 1
    off = hidden * cin * 27 + hidden + hidden * hidden * 27 + hidden
    m = np.zeros(n, dtype=np.uint8)
    for k in channels:
        if taps == "centre":
            m[off + k * 27 + TAP_CENTRE] = 1
        else:
            m[off + k * 27: off + (k + 1) * 27] = 1
    return m


def new_feature_closure(cfg: PairConfig, max_points: int, scale_seed: int = 10, stream=None) -> Closure:
    """A feature-input closure that starts as the modified-equation correction (biases zero, frozen)."""
    scales = feature_scales(scale_seed, cfg)
    probe = FineCoarsePair(scale_seed, cfg)
    kref = kappa_ref(probe)
    probe.close()
    t = 90.0 * scales[4] / kref  # makes the f4 pass-through weight of layer 3 equal to a
    cl = Closure(max_points, 1.0, cin=8, stream=stream)
    cl.set_features(FEATURE_SPACE_ORDER, scales)
    cl.set_out_scale(t)
    cl.freeze_biases(True)
    cl.set_params(modified_equation_params(scales, t, kref))
    cl.kref = kref
    return cl


def restricted_trajectory(pair: "FineCoarsePair", n_from: int, steps: int) -> dict:
    """Restricted fine levels n_from - 1 .. steps (dense FP32 CUDA tensors), keyed by coarse step."""
    out = {}
    for n in range(steps):
        pair.fine.run(2)
        if n + 1 >= n_from - 1:
            out[n + 1] = pair.restrict()
    return out


def train_rollout(closure: Closure, seeds, cfg: PairConfig, window: int = 25, n_from: int = 200, epochs: int = 2,
                  lr: float = 3e-3, lr_final: float = None, trainable="centre", log=None):
    """Train on coarse-grid rollouts: for windows [n0, n0 + window) with n0 >= n_from, start the
    corrected coarse grid from the restricted fine levels (n0, n0 - 1), take `window` corrected
    steps, and descend the mean relative squared error against the restricted fine levels
    (gradient by backpropagation through the steps, in the library).  Returns the losses.

    trainable: "centre" or "all" trains only the last layer's weights from the four
    modified-equation pass-through channels (their centre taps, or all 27 taps); None trains
    every weight.  (Training every weight makes Adam move the twelve free hidden channels by
    about lr per step, corrections far larger than the physical one, and the rollouts
    diverged; measured.)"""
    if trainable is None:
        N.closure_set_trainable(closure.h, None)
    else:
        N.closure_set_trainable(closure.h, output_weight_mask(taps=trainable))
    losses = []
    t0 = time.time()
    nwin = len(range(n_from, cfg.steps - window + 1, window))
    total = max(1, epochs * len(seeds) * nwin)
    lr_final = lr / 10 if lr_final is None else lr_final
    trajs = {}
    for sd in seeds:
        pair = FineCoarsePair(sd, cfg, stream=closure.stream)
        trajs[sd] = (restricted_trajectory(pair, n_from, cfg.steps), pair)
    k = 0
    for ep in range(epochs):
        for sd in seeds:
            ref, pair = trajs[sd]
            g = pair.coarse
            N.stencil_attach_closure(g.h, closure.h, C_REF)
            for n0 in range(n_from, cfg.steps - window + 1, window):
                refs = [ref[n0 + j + 1].data_ptr() for j in range(window)]
                L = N.stencil_closure_rollout_grad(g.h, ref[n0].data_ptr(), ref[n0 - 1].data_ptr(), n0, refs)
                closure.adam_step(lr * (lr_final / lr) ** (k / total))
                losses.append(L)
                k += 1
            N.stencil_attach_closure(g.h, None, C_REF)
            if log:
                log(f"epoch {ep} seed {sd}: {len(losses)} updates, last loss {losses[-1]:.3e}, "
                    f"{time.time() - t0:.1f}s")
    for sd in seeds:
        trajs[sd][1].close()
    return losses
