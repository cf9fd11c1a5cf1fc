"""Seeded synthetic XPCS speckle: AR(1) complex-Gaussian fields, Poisson counts, q-masks.

Workload model (the paper's experimental datasets are not available, so these inputs
stand in for them, with the shapes of the paper's workloads, Sec. 3):

* Every pixel p carries one complex-Gaussian speckle field E_p(t) with unit mean
  intensity.  E_p(0) ~ CN(0, 1) and E_p(t+1) = rho_p E_p(t) + sqrt(1 - rho_p^2) xi,
  xi ~ CN(0, 1), with rho_p = exp(-Gamma_p) and Gamma_p = D q_p^2 per frame, q_p the
  pixel's distance from the detector centre in pixels.  The field correlation is
  therefore g1(tau) = exp(-Gamma tau) and, for one mode per pixel, the Siegert relation
  gives g2(tau) - 1 = exp(-2 Gamma tau), the form of the relaxation in Eq. 13.
* The intensity is I = mean * |E|^2 and the count is Poisson(I), saturated at the
  maximum of the output dtype.

Two backends draw the same model: ``speckle_counts`` (numpy, Philox bit generator,
host memory, for the small cases the oracle handles) and ``speckle_counts_torch``
(torch generator on any device, for the full-size workloads).  They are separate
random streams; parity tests always feed the same bytes to both sides, so nothing
depends on the two backends agreeing draw by draw.

Nothing here computes a correlation: this module only makes inputs.
"""
from __future__ import annotations

import math

import numpy as np


def pixel_radius(H: int, W: int) -> np.ndarray:
    """Distance of each pixel centre from the detector centre, row-major (y * W + x)."""
    cy, cx = (H - 1) / 2.0, (W - 1) / 2.0
    y, x = np.mgrid[0:H, 0:W]
    return np.hypot(y - cy, x - cx).reshape(-1)


def ring_qmap(H: int, W: int, n_q: int) -> np.ndarray:
    """Equal-width rings about the centre: label = min(floor(r * n_q / r_max), n_q - 1).

    r_max is the farthest pixel centre, so every pixel gets a label in [0, n_q).
    """
    r = pixel_radius(H, W)
    rmax = r.max()
    lab = np.floor(r * n_q / rmax).astype(np.int64)
    return np.minimum(lab, n_q - 1).astype(np.int32)


def sector_qmap(H: int, W: int, n_annuli: int = 8, n_sectors: int = 8,
                min_px: int = 100, max_px: int = 20000, seed: int = 0) -> np.ndarray:
    """Ring-plus-angular-sector masks with log-spaced, uneven pixel counts.

    The n = n_annuli * n_sectors target sizes are round(min_px * (max_px/min_px)^(m/(n-1))).
    A seeded shuffle deals them to annuli (n_sectors each).  Pixels sorted by radius are
    cut into consecutive annuli whose sizes are the sums of their targets; each annulus,
    sorted by angle, is cut into its sectors.  Pixels left over get label -1.
    """
    n = n_annuli * n_sectors
    sizes = np.array([int(round(min_px * (max_px / min_px) ** (m / (n - 1)))) for m in range(n)])
    rng = np.random.Generator(np.random.Philox(seed))
    order = rng.permutation(n)
    groups = order.reshape(n_annuli, n_sectors)
    r = pixel_radius(H, W)
    if sizes.sum() > r.size:
        raise ValueError("detector too small for the requested mask sizes")
    cy, cx = (H - 1) / 2.0, (W - 1) / 2.0
    yy, xx = np.mgrid[0:H, 0:W]
    ang = np.arctan2(yy - cy, xx - cx).reshape(-1)
    by_r = np.argsort(r, kind="stable")
    qmap = np.full(r.size, -1, dtype=np.int32)
    pos = 0
    for a in range(n_annuli):
        labels = groups[a]
        tot = int(sizes[labels].sum())
        ann = by_r[pos:pos + tot]
        pos += tot
        ann = ann[np.argsort(ang[ann], kind="stable")]
        s = 0
        for lab in labels:
            qmap[ann[s:s + sizes[lab]]] = lab
            s += sizes[lab]
    return qmap


def rate_of_pixels(H: int, W: int, D: float) -> np.ndarray:
    """Per-pixel decay rate Gamma_p = D * q_p^2 (frames^-1), q_p in pixels."""
    r = pixel_radius(H, W)
    return D * r * r


def _dtype_max(dtype) -> int:
    return int(np.iinfo(np.dtype(dtype)).max)


def speckle_counts(H: int, W: int, T: int, mean: float, D: float, seed: int,
                   dtype=np.uint8, t0: int = 0) -> np.ndarray:
    """T x (H*W) photon counts from the AR(1) speckle model (numpy, host memory)."""
    M = H * W
    rho = np.exp(-rate_of_pixels(H, W, D))
    sig = np.sqrt(np.maximum(0.0, 1.0 - rho * rho))
    rng = np.random.Generator(np.random.Philox(seed))
    inv = 1.0 / math.sqrt(2.0)
    E = (rng.standard_normal(M) + 1j * rng.standard_normal(M)) * inv
    out = np.empty((T, M), dtype=dtype)
    cap = _dtype_max(dtype)
    for t in range(t0 + T):
        if t > 0:
            xi = (rng.standard_normal(M) + 1j * rng.standard_normal(M)) * inv
            E = rho * E + sig * xi
        if t >= t0:
            lam = mean * (E.real * E.real + E.imag * E.imag)
            out[t - t0] = np.minimum(rng.poisson(lam), cap).astype(dtype)
    return out


class TorchSpeckle:
    """Frame-by-frame AR(1) speckle generator on a torch device (for large workloads).

    ``next(n)`` returns the next n frames as an (n, H*W) uint8/uint16 tensor on the device.
    """

    def __init__(self, H: int, W: int, mean: float, D: float, seed: int,
                 dtype: str = "uint16", device: str = "cuda"):
        import torch

        self.torch = torch
        self.M = H * W
        self.mean = float(mean)
        self.device = torch.device(device)
        self.gen = torch.Generator(device=self.device)
        self.gen.manual_seed(int(seed))
        rho = torch.from_numpy(np.exp(-rate_of_pixels(H, W, D))).to(torch.float32)
        self.rho = rho.to(self.device)
        self.sig = torch.sqrt(torch.clamp(1.0 - self.rho * self.rho, min=0.0))
        inv = 1.0 / math.sqrt(2.0)
        self.er = torch.randn(self.M, generator=self.gen, device=self.device) * inv
        self.ei = torch.randn(self.M, generator=self.gen, device=self.device) * inv
        self.started = False
        self.tdtype = {"uint8": torch.uint8, "uint16": torch.uint16}[dtype]
        self.cap = 255 if dtype == "uint8" else 65535

    def next(self, n: int):
        torch = self.torch
        out = torch.empty((n, self.M), dtype=self.tdtype, device=self.device)
        inv = 1.0 / math.sqrt(2.0)
        for i in range(n):
            if self.started:
                xr = torch.randn(self.M, generator=self.gen, device=self.device)
                xi = torch.randn(self.M, generator=self.gen, device=self.device)
                self.er.mul_(self.rho).add_(xr.mul_(self.sig * inv))
                self.ei.mul_(self.rho).add_(xi.mul_(self.sig * inv))
            self.started = True
            lam = (self.er * self.er + self.ei * self.ei).mul_(self.mean)
            cnt = torch.poisson(lam, generator=self.gen).clamp_(max=self.cap)
            out[i].copy_(cnt.to(torch.int32))
        return out


def speckle_counts_torch(H: int, W: int, T: int, mean: float, D: float, seed: int,
                         dtype: str = "uint16", device: str = "cuda"):
    """T x (H*W) photon counts from the AR(1) speckle model, drawn on a torch device."""
    return TorchSpeckle(H, W, mean, D, seed, dtype=dtype, device=device).next(T)
