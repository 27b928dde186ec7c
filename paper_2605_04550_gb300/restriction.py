"""Learned restriction of the sigma_min evaluation: the hybrid method of the
paper (Sec. 3-4) on the library's kernels.

1. Features (psa_matrix_stats, psa_global_features, psa_point_features): global
   matrix features and per-point features, one BF16 row per grid point.
2. Labels: sensitive iff sigma_min(zI - A) <= eps (Sec. 2.1), computed by the
   plain GPU method (batched sigma_min) on the training matrices' grids.
3. Training (psa_mlp_train_step): balanced sampling of the labelled points
   (Sec. 3.3.1), Adam on binary cross-entropy, batch 512, up to 25 epochs with
   early stopping on a held-out loss (Sec. 3.4).
4. Hierarchical prediction (Sec. 3.5): the network on the stride-4 coarse grid,
   then on the 4 x 4 fine points of the flagged coarse cells; other points get
   probability 0.
5. Calibration (Sec. 3.6): the decision threshold tau chosen on validation
   matrices from recall against 3 x 3-dilated truth with 5 x 5-dilated
   predictions; here the largest tau whose smallest validation recall is at
   least the target (0.99).
6. Restricted run (Sec. 4): R = dilate_5x5(p >= tau), exact sigma_min on R only
   (psa_sigma_min with the point list in tile order); all other points are
   classified non-sensitive.

Host code here only marshals arguments, draws sample indices and keeps
bookkeeping; every pass over matrix or grid data runs in the library's kernels.
"""
from __future__ import annotations

import ctypes
import dataclasses
import time
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import LanczosOpts, _native, batch, mlp, sigma_min
from .inputs import Grid

EPS = 1e-2
TARGET_RECALL = 0.99
# labels decide sigma <= eps: a relative accuracy of about 1e-6 on sigma settles every
# point farther than that from the level; the resolvent-norm features need ~3 digits
LABEL_OPTS = LanczosOpts(k_min=2, k_max=1000, tol=1e-6)
PROBE_OPTS = LanczosOpts(k_min=2, k_max=300, tol=1e-6)
BATCH_STREAMS = 8


def _grid_c(g: Grid) -> _native.PsaGrid:
    return _native.PsaGrid(float(g.re_min), float(g.re_max), float(g.im_min), float(g.im_max), int(g.nx), int(g.ny))


@dataclasses.dataclass
class MatrixContext:
    """Device-resident features of one matrix."""
    bands: object   # CUDA complex128 (kl + ku + 1, n)
    kl: int
    ku: int
    stats: object   # CUDA float64 [STATS]
    symbol: object  # CUDA complex128 [SYMBOL_SAMPLES]
    glob: object    # CUDA float32 [GLOBAL_FEATURES]
    #: CUDA complex128 [m]: a point set (the eigenvalues of A) that replaces the symbol
    #: curve in the spectrum features, or None (the symbol curve)
    spectrum: object = None


def matrix_contexts(mats: Sequence[Tuple[object, int, int]], eps: float = EPS,
                    opts: Optional[LanczosOpts] = None, spectra: Optional[Sequence[object]] = None
                    ) -> List[MatrixContext]:
    """Global features of every matrix (bands already on the device). The four
    sigma_min probes (z = 0 and the centroid + 0.5, 1, 2) of all matrices run as
    one batched call. With ``spectra`` (one array of eigenvalues per matrix, host
    or device), the spectrum features are the paper's own, taken over those
    eigenvalues instead of the symbol curve (psa_point_set_stats)."""
    import torch
    lib = _native.load()
    dev = mats[0][0].device
    s = torch.cuda.current_stream(dev)
    stats = torch.empty((len(mats), _native.STATS), dtype=torch.float64, device=dev)
    symbol = torch.empty((len(mats), _native.SYMBOL_SAMPLES), dtype=torch.complex128, device=dev)
    if spectra is not None and len(spectra) != len(mats):
        raise ValueError("one eigenvalue array per matrix")
    sets = [None] * len(mats)
    for m, (b, kl, ku) in enumerate(mats):
        A = _native.PsaBand(int(b.shape[1]), int(kl), int(ku), b.data_ptr())
        _native.check(lib.psa_matrix_stats(ctypes.byref(A), stats[m].data_ptr(), symbol[m].data_ptr(), s.cuda_stream),
                      "psa_matrix_stats")
        if spectra is not None:
            sets[m] = torch.as_tensor(spectra[m], dtype=torch.complex128, device=dev).reshape(-1).contiguous()
            if sets[m].numel() < 1 or sets[m].numel() > 2**31 - 1:
                raise ValueError("an eigenvalue array must hold 1 to 2^31 - 1 values")
            _native.check(lib.psa_point_set_stats(sets[m].data_ptr(), int(sets[m].numel()), stats[m].data_ptr(),
                                                  s.cuda_stream), "psa_point_set_stats")
    cen = stats[:, :2].cpu().numpy()  # the probe grids are host arguments
    entries = []
    for m, (b, kl, ku) in enumerate(mats):
        cr, ci = float(cen[m, 0]), float(cen[m, 1])
        entries.append((b, kl, ku, Grid(0.0, 0.0, 0.0, 0.0, 1, 1)))
        entries.append((b, kl, ku, Grid(cr + 0.5, cr + 2.0, ci, ci, 4, 1)))
    plan = batch.BatchPlan(entries)
    o = opts or PROBE_OPTS
    r = batch.sigma_min_batched(plan, (), o, workspace=_workspace(plan, o),
                                config=batch.BatchConfig(streams=BATCH_STREAMS))
    sig = r.sigma.view(len(mats), 5)
    sigma4 = torch.stack([sig[:, 0], sig[:, 1], sig[:, 2], sig[:, 4]], dim=1).contiguous()
    glob = torch.empty((len(mats), _native.GLOBAL_FEATURES), dtype=torch.float32, device=dev)
    for m in range(len(mats)):
        _native.check(lib.psa_global_features(stats[m].data_ptr(), sigma4[m].data_ptr(), float(eps),
                                              glob[m].data_ptr(), s.cuda_stream), "psa_global_features")
    return [MatrixContext(b, kl, ku, stats[m], symbol[m], glob[m], sets[m]) for m, (b, kl, ku) in enumerate(mats)]


def point_features(ctx: MatrixContext, grid: Grid, idx=None, out=None):
    """BF16 feature rows (npoints, IN) of the grid's points (or of the flat indices idx)."""
    import torch
    lib = _native.load()
    dev = ctx.bands.device
    n = grid.npoints if idx is None else int(idx.numel())
    x = out if out is not None else torch.empty((n, mlp.IN), dtype=torch.bfloat16, device=dev)
    if n == 0:
        return x  # an empty list (a NULL list would mean the full grid)
    if idx is not None and (idx.dtype != torch.int32 or not idx.is_contiguous() or idx.device != dev):
        raise TypeError("idx must be a contiguous int32 tensor on the bands' device")
    if x.shape != (n, mlp.IN) or x.dtype != torch.bfloat16 or not x.is_contiguous():
        raise ValueError("out must be a contiguous bfloat16 (npoints, IN) tensor")
    g = _grid_c(grid)
    s = torch.cuda.current_stream(dev)
    ip, ni = (idx.data_ptr(), n) if idx is not None else (None, 0)
    if ctx.spectrum is None:
        _native.check(lib.psa_point_features(ctypes.byref(g), ip, ni, ctx.stats.data_ptr(), ctx.symbol.data_ptr(),
                                             ctx.glob.data_ptr(), x.data_ptr(), s.cuda_stream), "psa_point_features")
    else:
        _native.check(lib.psa_point_features_set(ctypes.byref(g), ip, ni, ctx.stats.data_ptr(),
                                                 ctx.spectrum.data_ptr(), int(ctx.spectrum.numel()), 0,
                                                 ctx.glob.data_ptr(), x.data_ptr(), s.cuda_stream),
                      "psa_point_features_set")
    return x


def region_mask(prob, grid: Grid, tau: float, radius: int = 2):
    """uint8 (ny, nx): dilate_{(2 radius + 1)^2}({p >= tau})."""
    import torch
    lib = _native.load()
    if prob.dtype != torch.float32 or not prob.is_cuda or not prob.is_contiguous() or prob.numel() != grid.npoints:
        raise ValueError("prob must be a contiguous CUDA float32 tensor with one value per grid point")
    out = torch.empty((grid.ny, grid.nx), dtype=torch.uint8, device=prob.device)
    _native.check(lib.psa_region(prob.data_ptr(), float(tau), grid.nx, grid.ny, int(radius), out.data_ptr(),
                                 torch.cuda.current_stream(prob.device).cuda_stream), "psa_region")
    return out


def region_list(mask, grid: Grid):
    """Flat indices (CUDA int32) of a mask's points in tile order (the restricted list)."""
    import torch
    lib = _native.load()
    if mask.dtype != torch.uint8 or not mask.is_cuda or not mask.is_contiguous() or mask.numel() != grid.npoints:
        raise ValueError("mask must be a contiguous CUDA uint8 tensor with one value per grid point")
    slots = torch.empty(((grid.nx + 7) // 8) * ((grid.ny + 3) // 4) * 32, dtype=torch.int32, device=mask.device)
    _native.check(lib.psa_tile_slots(mask.data_ptr(), grid.nx, grid.ny, slots.data_ptr(),
                                     torch.cuda.current_stream(mask.device).cuda_stream), "psa_tile_slots")
    return slots[slots >= 0].contiguous()


def _workspace(plan, opts, cap_bytes: float = 64e9):
    return batch.BatchWorkspace(plan, opts, max_bytes=int(cap_bytes), streams=BATCH_STREAMS)


def labels_batched(mats, grids, eps: float = EPS, opts: LanczosOpts = LABEL_OPTS, with_status: bool = False):
    """sigma_min on every grid (one batched call): returns (plan, sigma flat CUDA float64
    [, status])."""
    plan = batch.BatchPlan([(b, kl, ku, g) for (b, kl, ku), g in zip(mats, grids)])
    r = batch.sigma_min_batched(plan, (eps,), opts, workspace=_workspace(plan, opts),
                                config=batch.BatchConfig(streams=BATCH_STREAMS))
    return (plan, r.sigma, r.status) if with_status else (plan, r.sigma)


def dilate_np(mask: np.ndarray, radius: int) -> np.ndarray:
    """Box dilation of a small boolean array (metrics bookkeeping on the host)."""
    m = np.asarray(mask, dtype=bool)
    ny, nx = m.shape
    p = np.zeros((ny + 2 * radius, nx + 2 * radius), dtype=bool)
    p[radius:radius + ny, radius:radius + nx] = m
    out = np.zeros_like(m)
    for a in range(2 * radius + 1):
        for b in range(2 * radius + 1):
            out |= p[a:a + ny, b:b + nx]
    return out


def recall_metrics(truth: np.ndarray, pred_region: np.ndarray) -> dict:
    """Paper Sec. 5.2: recall against 3 x 3-dilated truth, coverage against truth,
    precision, grid fraction."""
    t = np.asarray(truth, dtype=bool)
    r = np.asarray(pred_region, dtype=bool)
    td = dilate_np(t, 1)
    rec = float((td & r).sum() / td.sum()) if td.any() else 1.0
    cov = float((t & r).sum() / t.sum()) if t.any() else 1.0
    prec = float((t & r).sum() / r.sum()) if r.any() else 1.0
    return {"recall": rec, "coverage": cov, "precision": prec, "grid_fraction": float(r.mean()),
            "sensitive_fraction": float(t.mean())}


#: column of a feature row holding log10(distance to the symbol polyline, or to the
#: nearest eigenvalue with eigenvalue features, / eps)
NEAR_COL = 32 + _native.GLOBAL_FEATURES
#: points within NEAR_FACTOR * eps of the symbol curve always enter the region
NEAR_FACTOR = 2.0


def near_curve(x, grid: Grid, eps: float, coarse: bool = False):
    """Boolean (rows,) from feature rows x: the point lies within NEAR_FACTOR * eps of the
    symbol curve (for a coarse anchor of the hierarchical pass: within that band plus
    the reach of its 4 x 4 cell). For banded Toeplitz-like A the curve itself lies in
    Lambda_eps once n is large (sigma_min(zI - A) -> 0 on it), and sigma_min is
    1-Lipschitz in z, so these points are sensitive or next to the zone; the rule
    catches the thin zone of nearly normal matrices (a kl = ku Grcar-type band), which
    is a band of width 2 eps about the spectrum that coarse training labels rarely hit.
    With eigenvalue features the column holds the distance to the nearest eigenvalue,
    and sigma_min(zI - A) <= |z - lambda| for every eigenvalue lambda."""
    h = max((grid.re_max - grid.re_min) / max(grid.nx - 1, 1), (grid.im_max - grid.im_min) / max(grid.ny - 1, 1))
    reach = NEAR_FACTOR * eps + (4.25 * h if coarse else 0.0)
    return x[:, NEAR_COL].float() <= float(np.log10(reach / eps))


def _grow(flag):
    """Flagged coarse cells plus their 8 neighbours: a cell whose own anchor falls just
    outside the zone still gets its fine points evaluated when a neighbouring anchor
    is flagged (the coarse counterpart of the 5 x 5 safety dilation)."""
    import torch
    f = flag.to(torch.float32)[None, None]
    return torch.nn.functional.max_pool2d(f, 3, stride=1, padding=1)[0, 0] > 0


class Restriction:
    """The trained classifier with its calibrated thresholds."""

    def __init__(self, device="cuda", seed: int = 0, eps: float = EPS, net: str = "mlp",
                 features: str = "symbol"):
        if features not in ("symbol", "eigen"):
            raise ValueError("features must be 'symbol' (the symbol curve) or 'eigen' (eigenvalues)")
        self.net = net
        self.features = features
        self.theta = mlp.init_theta(seed, device, net)
        self.device = device
        self.eps = eps
        self.tau = 0.5
        self.history = []
        self.calibration = {}

    # ---------------------------------------------------------- persistence
    def save(self, path: str, meta: Optional[dict] = None):
        """Parameters, threshold and calibration summary to an .npz file."""
        import json
        th = self.theta.detach().cpu().numpy().astype(np.float32)
        info = {"tau": self.tau, "eps": self.eps, "net": self.net, "features": self.features, "meta": meta or {},
                "calibration": {k: v for k, v in self.calibration.items() if k != "table"}}
        np.savez(path, theta=th, info=np.frombuffer(json.dumps(info).encode(), dtype=np.uint8))

    @classmethod
    def load(cls, path: str, device="cuda"):
        import json
        import torch
        d = np.load(path)
        th = d["theta"]
        info = json.loads(bytes(d["info"]).decode())
        net = info.get("net", "mlp")
        if th.shape != (mlp.nparam(net),) or th.dtype != np.float32:
            raise ValueError("parameter vector of the wrong size")
        r = cls(device, eps=float(info["eps"]), net=net, features=info.get("features", "symbol"))
        r.theta = torch.as_tensor(th, device=device)
        r.tau = float(info["tau"])
        r.calibration = info.get("calibration", {})
        r.meta = info.get("meta", {})
        return r

    # ------------------------------------------------------------ training
    def build_training_set(self, mats, grids, rng: np.random.Generator, opts: LanczosOpts = LABEL_OPTS,
                           spectra=None, labels=None):
        """Features and labels of the training matrices, balanced per matrix: all
        positives and max(10 n_pos, 200) negatives (fewer if the grid has fewer).
        ``spectra``: the eigenvalues of each matrix, for a classifier on eigenvalue
        features. ``labels``: the ``last_labels`` of an earlier call on the same
        matrices and grids, to reuse its sigma_min labels (with an rng in the same
        state the same points are drawn)."""
        import torch
        if (spectra is not None) != (self.features == "eigen"):
            raise ValueError("spectra are required exactly for a classifier on eigenvalue features")
        dev = mats[0][0].device
        t0 = time.perf_counter()
        ctxs = matrix_contexts(mats, self.eps, spectra=spectra)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        if labels is None:
            plan, sig, st = labels_batched(mats, grids, self.eps, opts, with_status=True)
            offsets = list(plan.offsets)
            lab = (sig <= self.eps).to(torch.uint8).cpu().numpy()
            stc = np.bincount(st.cpu().numpy().astype(np.int64), minlength=6)
            counts = {str(k): int(v) for k, v in enumerate(stc) if v}
        else:
            offsets, lab, counts = labels
        self.last_labels = (offsets, lab, counts)
        t2 = time.perf_counter()
        self.timing = {"contexts_s": t1 - t0, "labels_s": t2 - t1, "label_points": int(lab.size),
                       "label_status_counts": counts}
        xs, ys = [], []
        for m, (ctx, g) in enumerate(zip(ctxs, grids)):
            o = offsets[m]
            y = lab[o:o + g.npoints]
            pos = np.flatnonzero(y)
            neg = np.flatnonzero(y == 0)
            k = min(neg.size, max(10 * pos.size, 200))
            pick = np.concatenate([pos, rng.choice(neg, k, replace=False)]) if k else pos
            x = point_features(ctx, g)
            sel = torch.as_tensor(pick, device=x.device)
            xs.append(x.index_select(0, sel))
            ys.append(torch.as_tensor(y[pick].astype(np.float32), device=x.device))
        xs, ys = torch.cat(xs), torch.cat(ys)
        torch.cuda.synchronize(dev)
        self.timing["features_s"] = time.perf_counter() - t2
        self.timing["samples"] = int(ys.numel())
        self.timing["positive_fraction"] = float(ys.mean().item())
        return xs, ys, ctxs

    def train(self, x, y, rng: np.random.Generator, epochs: int = 25, patience: int = 5, batch: int = 512,
              lr: float = 1e-3, holdout: float = 0.1, log=None):
        """Adam on BCE; the held-out fraction gives the early-stopping loss."""
        import torch
        S = x.shape[0]
        perm = torch.as_tensor(rng.permutation(S), device=x.device)
        nv = max(int(S * holdout), 1)
        xv, yv = x.index_select(0, perm[:nv]), y.index_select(0, perm[:nv])
        xt, yt = x.index_select(0, perm[nv:]), y.index_select(0, perm[nv:])
        tr = mlp.Trainer(self.theta, batch=batch, lr=lr, net=self.net)
        best, best_theta, bad = float("inf"), self.theta.clone(), 0
        yv_np = yv.cpu().numpy()
        for ep in range(epochs):
            t0 = time.perf_counter()
            order = torch.as_tensor(rng.permutation(xt.shape[0]), device=x.device)
            nb = xt.shape[0] // batch
            for b in range(nb):
                sel = order[b * batch:(b + 1) * batch]
                tr.step(xt.index_select(0, sel), yt.index_select(0, sel))
            p = mlp.forward(self.theta, xv, net=self.net).cpu().numpy().astype(np.float64)
            mlp.check_timeouts()  # the epoch's GEMMs all completed their waits
            p = np.clip(p, 1e-7, 1 - 1e-7)
            vloss = float(-np.mean(yv_np * np.log(p) + (1 - yv_np) * np.log(1 - p)))
            self.history.append({"epoch": ep, "val_loss": vloss, "seconds": time.perf_counter() - t0,
                                 "val_acc": float(np.mean((p >= 0.5) == (yv_np > 0.5)))})
            if log:
                log(self.history[-1])
            if vloss < best - 1e-6:
                best, best_theta, bad = vloss, self.theta.clone(), 0
            else:
                bad += 1
                if bad >= patience:
                    break
        self.theta.copy_(best_theta)
        return self.history

    # ----------------------------------------------------------- inference
    def _check_ctx(self, ctx: MatrixContext):
        if (ctx.spectrum is not None) != (self.features == "eigen"):
            raise ValueError(f"this classifier takes {self.features} features; build the context "
                             + ("with spectra=" if self.features == "eigen" else "without spectra"))

    def predict(self, ctx: MatrixContext, grid: Grid, hierarchical: bool = True, tau: Optional[float] = None):
        """Probability map (ny, nx) float32 on the device. Hierarchical: the coarse
        stride-4 grid first; a coarse cell is refined (its 4 x 4 fine points
        evaluated) when its probability, or that of a neighbouring coarse cell,
        reaches the 80th percentile of the coarse map or the decision threshold,
        whichever is lower; other points get 0."""
        import torch
        self._check_ctx(ctx)
        dev = ctx.bands.device
        nx, ny = grid.nx, grid.ny
        if not hierarchical:
            x = point_features(ctx, grid)
            p = mlp.forward(self.theta, x, net=self.net)
            return torch.where(near_curve(x, grid, self.eps), torch.ones_like(p), p).view(ny, nx)
        ic = torch.arange(0, ny, 4, device=dev, dtype=torch.int32)
        jc = torch.arange(0, nx, 4, device=dev, dtype=torch.int32)
        cidx = (ic[:, None] * nx + jc[None, :]).reshape(-1).contiguous()
        xc = point_features(ctx, grid, cidx)
        pc = mlp.forward(self.theta, xc, net=self.net)
        t = self.tau if tau is None else tau
        tc = min(float(torch.quantile(pc.float(), 0.8).item()), t)
        flag = _grow(((pc >= tc) | near_curve(xc, grid, self.eps, coarse=True)).view(ic.numel(), jc.numel()))
        # fine points of flagged cells
        fi = (ic[:, None] + torch.arange(4, device=dev, dtype=torch.int32)[None, :])  # (nyc, 4)
        fj = (jc[:, None] + torch.arange(4, device=dev, dtype=torch.int32)[None, :])  # (nxc, 4)
        cells = flag.nonzero()
        ii = fi[cells[:, 0]][:, :, None].expand(-1, 4, 4)
        jj = fj[cells[:, 1]][:, None, :].expand(-1, 4, 4)
        ok = (ii < ny) & (jj < nx)
        fidx = (ii * nx + jj)[ok].to(torch.int32).contiguous()
        prob = torch.zeros(ny * nx, dtype=torch.float32, device=dev)
        if fidx.numel():
            xf = point_features(ctx, grid, fidx)
            pf = mlp.forward(self.theta, xf, net=self.net)
            prob[fidx.long()] = torch.where(near_curve(xf, grid, self.eps), torch.ones_like(pf), pf)
        self.last_counts = {"coarse": int(cidx.numel()), "fine": int(fidx.numel()), "tau_coarse": tc}
        return prob.view(ny, nx)

    # ---------------------------------------------------------- calibration
    @staticmethod
    def hierarchical_mask(full, tau: float, near_coarse=None):
        """The hierarchical map from the full fine map (the network gives every point
        the same value alone or in any batch): coarse points are full[::4, ::4];
        fine values survive in the 4 x 4 cells whose coarse value reaches
        min(80th percentile, tau) or whose anchor is near the curve (near_coarse),
        and their neighbours; zero elsewhere."""
        import torch
        pc = full[::4, ::4]
        tc = min(float(torch.quantile(pc.reshape(-1).float(), 0.8).item()), tau)
        flag = pc >= tc
        if near_coarse is not None:
            flag = flag | near_coarse
        keep = _grow(flag).repeat_interleave(4, 0).repeat_interleave(4, 1)[:full.shape[0], :full.shape[1]]
        return torch.where(keep, full, torch.zeros_like(full))

    def coarse_near(self, ctx: MatrixContext, grid: Grid):
        """near_curve of the hierarchical pass's coarse anchors, as a (ny/4, nx/4) map."""
        import torch
        dev = ctx.bands.device
        ic = torch.arange(0, grid.ny, 4, device=dev, dtype=torch.int32)
        jc = torch.arange(0, grid.nx, 4, device=dev, dtype=torch.int32)
        cidx = (ic[:, None] * grid.nx + jc[None, :]).reshape(-1).contiguous()
        xc = point_features(ctx, grid, cidx)
        return near_curve(xc, grid, self.eps, coarse=True).view(ic.numel(), jc.numel())

    def calibrate(self, ctxs, grids, sig_truth: List[np.ndarray], taus=None, hierarchical: bool = True,
                  target: float = TARGET_RECALL):
        """Largest tau whose smallest recall over the validation matrices reaches the
        target; also the paper's literal rule (smallest tau with median recall >= 0.9
        and 10th-percentile recall >= 0.75) for reference."""
        import torch
        if taus is None:
            taus = list(np.round(np.arange(0.001, 0.01, 0.001), 3)) + list(np.round(np.arange(0.01, 1.0, 0.01), 2))
        taus = list(taus)
        full = [self.predict(c, g, hierarchical=False) for c, g in zip(ctxs, grids)]
        nearc = [self.coarse_near(c, g) for c, g in zip(ctxs, grids)]
        table, per_matrix = [], []
        for t in taus:
            recs, fracs, recs_full = [], [], []
            for pf, nc, g, s in zip(full, nearc, grids, sig_truth):
                p = self.hierarchical_mask(pf, t, nc) if hierarchical else pf
                r = region_mask(p.reshape(-1).contiguous(), g, t).cpu().numpy().astype(bool)
                mtr = recall_metrics(s <= self.eps, r)
                recs.append(mtr["recall"])
                fracs.append(mtr["grid_fraction"])
                rf = region_mask(pf.reshape(-1).contiguous(), g, t).cpu().numpy().astype(bool)
                recs_full.append(recall_metrics(s <= self.eps, rf)["recall"])
            per_matrix.append(recs)
            table.append({"tau": float(t), "min_recall": float(np.min(recs)), "median_recall": float(np.median(recs)),
                          "p10_recall": float(np.percentile(recs, 10)), "mean_grid_fraction": float(np.mean(fracs)),
                          "min_recall_without_hierarchy": float(np.min(recs_full))})
        ok = [row for row in table if row["min_recall"] >= target]
        chosen = max(ok, key=lambda r: r["tau"]) if ok else min(table, key=lambda r: r["tau"])
        paper = [row for row in table if row["median_recall"] >= 0.9 and row["p10_recall"] >= 0.75]
        self.tau = chosen["tau"]
        recs = per_matrix[taus.index(chosen["tau"])]
        self.calibration = {"tau": self.tau, "target_recall": target, "row": chosen,
                            "paper_rule_tau": min(r["tau"] for r in paper) if paper else None,
                            "matrices": len(grids), "per_matrix_recall": [float(r) for r in recs],
                            "worst_matrix": int(np.argmin(recs)), "table": table}
        return self.calibration

    # --------------------------------------------------------- restricted run
    def restricted(self, ctx: MatrixContext, grid: Grid, eps: Sequence[float], opts: Optional[LanczosOpts] = None,
                   workspace=None, hierarchical: bool = True):
        """Classifier + region + exact sigma_min on the region only. Returns the
        sigma_min result (NOT_EVALUATED outside R), the region mask and timings."""
        import torch
        dev = ctx.bands.device
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        prob = self.predict(ctx, grid, hierarchical)
        mask = region_mask(prob.reshape(-1).contiguous(), grid, self.tau)
        idx = region_list(mask, grid)
        e[1].record()
        out = sigma_min(ctx.bands, ctx.kl, ctx.ku, grid, eps=eps, idx=idx, opts=opts, workspace=workspace)
        e[2].record()
        torch.cuda.synchronize(dev)
        return out, mask, idx, {"nn_ms": e[0].elapsed_time(e[1]), "restricted_ms": e[1].elapsed_time(e[2])}
