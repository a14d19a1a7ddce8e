"""Seeded synthetic SLC stacks (input generation only).

This module holds none of the phase-linking arithmetic: it draws inputs.  Tests
feed the same arrays to the CUDA path and to the CPU oracle; the benchmark
draws its full-size stacks with it directly on the GPU.

Pixel model (Sec. II-A): each pixel vector z is circular complex Gaussian with
unit power per date and coherence
    Gamma_ik = rho_inf + (rho0 - rho_inf) exp(-|t_i - t_k| / tau),  Gamma_ii = 1,
the exponential-decay model of Sec. II-C.  It is drawn without a per-pixel
Cholesky factor, by summing three independent circular Gaussian parts:
    z_i = exp(j phi_i) [ sqrt(rho_inf) c + sqrt(rho0 - rho_inf) a_i + sqrt(1 - rho0) n_i ]
where c is one draw shared by all dates, n_i are independent per date, and a_i
is a stationary Gauss-Markov sequence a_i = r_i a_{i-1} + sqrt(1 - r_i^2) w_i,
r_i = exp(-(t_i - t_{i-1}) / tau), whose correlation is exp(-|t_i - t_k| / tau).
The true phase history phi (a linear ramp, optionally with a step on a patch) is
carried as exp(+j phi_i), so Sigma_ik = E[z_i conj(z_k)] = Gamma_ik e^{j(phi_i - phi_k)}.
Amplitudes are Rayleigh.  Persistent-scatterer pixels are A0 e^{j phi_i}(1 + eps_i)
with eps_i ~ CN(0, sigma^2), which gives amplitude dispersion ~ sigma / sqrt(2).

All draws come from one torch.Generator on the target device, seeded, in a
fixed order, row chunk by row chunk; CPU and GPU streams differ, so a test that
compares the two paths draws once and copies.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch


@dataclass
class StackSpec:
    N: int
    H: int
    W: int
    rho0: float = 0.7
    rho_inf: float = 0.1
    tau: float | tuple[float, float] = 48.0   # days, or a per-pixel U(lo, hi) range
    dt: float = 12.0                          # days between acquisitions
    ramp: float = 0.05                        # rad per date
    ps_fraction: float = 0.0
    ps_amp: float = 3.0
    ps_sigma: float = 0.1
    # phase step: (first date index, row0, row1, col0, col1, rad) or None
    step: tuple | None = None
    # near-singular patches: (area fraction, patch size, rho) or None
    patches: tuple | None = None
    date_offset: int = 0                      # index of date 0 in the archive
    seed: int = 0
    extra: dict = field(default_factory=dict)


def true_phase(spec: StackSpec, rows: slice | None = None, cols: slice | None = None,
               device="cpu") -> torch.Tensor:
    """phi [N, h, w] (float64) of the stack, absolute (archive) date indexing."""
    r0, r1 = (0, spec.H) if rows is None else (rows.start, rows.stop)
    c0, c1 = (0, spec.W) if cols is None else (cols.start, cols.stop)
    t = torch.arange(spec.N, dtype=torch.float64, device=device) + spec.date_offset
    ph = (spec.ramp * t).view(-1, 1, 1).expand(spec.N, r1 - r0, c1 - c0).clone()
    if spec.step is not None:
        d0, sr0, sr1, sc0, sc1, rad = spec.step
        rr0, rr1 = max(sr0, r0), min(sr1, r1)
        cc0, cc1 = max(sc0, c0), min(sc1, c1)
        if rr0 < rr1 and cc0 < cc1:
            sel = t >= d0
            ph[sel, rr0 - r0:rr1 - r0, cc0 - c0:cc1 - c0] += rad
    return ph


def _cn(shape, gen, device):
    return torch.randn(shape, dtype=torch.complex64, generator=gen, device=device)


def _patch_map(spec: StackSpec, gen, device) -> torch.Tensor | None:
    if spec.patches is None:
        return None
    frac, size, _rho = spec.patches
    n = max(1, int(round(frac * spec.H * spec.W / (size * size))))
    m = torch.zeros(spec.H, spec.W, dtype=torch.bool, device=device)
    ys = torch.randint(0, max(1, spec.H - size), (n,), generator=gen, device=device).tolist()
    xs = torch.randint(0, max(1, spec.W - size), (n,), generator=gen, device=device).tolist()
    for y, x in zip(ys, xs):
        m[y:y + size, x:x + size] = True
    return m


@torch.no_grad()
def generate(spec: StackSpec, device="cpu", row_chunk: int = 256,
             out: torch.Tensor | None = None) -> torch.Tensor:
    """Draw the complex64 stack [N, H, W] of `spec` on `device`."""
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(spec.seed))
    N, H, W = spec.N, spec.H, spec.W
    if out is None:
        out = torch.empty((N, H, W), dtype=torch.complex64, device=dev)
    patch = _patch_map(spec, gen, dev)
    for r0 in range(0, H, row_chunk):
        r1 = min(H, r0 + row_chunk)
        h = r1 - r0
        if isinstance(spec.tau, tuple):
            lo, hi = spec.tau
            tau = lo + (hi - lo) * torch.rand((h, W), generator=gen, device=dev, dtype=torch.float32)
        else:
            tau = torch.full((h, W), float(spec.tau), device=dev, dtype=torch.float32)
        rho0 = torch.full((h, W), float(spec.rho0), device=dev)
        rinf = torch.full((h, W), float(spec.rho_inf), device=dev)
        if patch is not None:
            p = patch[r0:r1]
            rho0 = torch.where(p, torch.full_like(rho0, spec.patches[2]), rho0)
            rinf = torch.where(p, torch.full_like(rinf, spec.patches[2]), rinf)
        r = torch.exp(-spec.dt / tau)
        ar = torch.sqrt(1.0 - r * r)
        s_c = torch.sqrt(rinf)
        s_a = torch.sqrt(torch.clamp(rho0 - rinf, min=0.0))
        s_n = torch.sqrt(torch.clamp(1.0 - rho0, min=0.0))
        c = _cn((h, W), gen, dev)
        a = _cn((h, W), gen, dev)
        ps = None
        if spec.ps_fraction > 0:
            ps = torch.rand((h, W), generator=gen, device=dev) < spec.ps_fraction
        phi = true_phase(spec, slice(r0, r1), slice(0, W), device=dev).to(torch.float32)
        for i in range(N):
            if i > 0:
                a = r * a + ar * _cn((h, W), gen, dev)
            n = _cn((h, W), gen, dev)
            zi = s_c * c + s_a * a + s_n * n
            if ps is not None:
                eps = spec.ps_sigma * _cn((h, W), gen, dev)
                zi = torch.where(ps, spec.ps_amp * (1.0 + eps), zi)
            out[i, r0:r1] = zi * torch.polar(torch.ones_like(phi[i]), phi[i])
    return out


# --------------------------------------------------------------------------
# The five workloads (sizes, value distributions and structure of the paper's
# burst-shaped stacks).  `scale` shrinks the image for oracle-sized cases.
# --------------------------------------------------------------------------

def config_spec(cfg: int, scale: float = 1.0, **over) -> StackSpec:
    def sz(n):
        return max(1, int(round(n * scale)))
    if cfg == 0:   # N=10 x 128x128, rho 0.6 e^{-t/48} + 0.1, ramp 0.05, 11x5 stride 1
        s = StackSpec(N=10, H=sz(128), W=sz(128), rho0=0.7, rho_inf=0.1, tau=48.0, seed=0)
    elif cfg == 1:  # N=15 x 4096x16384 burst, tau ~ U(12,120), 5% PS, 11x5 strides 6x3
        s = StackSpec(N=15, H=sz(4096), W=sz(16384), rho0=0.7, rho_inf=0.1, tau=(12.0, 120.0),
                      ps_fraction=0.05, ps_amp=3.0, ps_sigma=0.1, seed=1)
    elif cfg == 2:  # one of 64 uneven stacks, 1024x2048; caller sets N, rho0 and seed
        s = StackSpec(N=15, H=sz(1024), W=sz(2048), rho0=0.6, rho_inf=0.1, tau=48.0,
                      patches=(0.01, 32, 0.98), seed=2)
    elif cfg == 3:  # 60 dates x 2048x4096, +2 rad from date 31 on a 200x200 patch
        H, W = sz(2048), sz(4096)
        p0y, p0x, pn = int(924 * scale), int(1948 * scale), max(1, int(200 * scale))
        s = StackSpec(N=60, H=H, W=W, rho0=0.7, rho_inf=0.1, tau=48.0,
                      step=(30, p0y, p0y + pn, p0x, p0x + pn, 2.0), seed=3)
    elif cfg == 4:  # N=20 x 1024x1024, coherence and ramp of the 128x128 stack
        s = StackSpec(N=20, H=sz(1024), W=sz(1024), rho0=0.7, rho_inf=0.1, tau=48.0, seed=4)
    else:
        raise ValueError(f"unknown workload {cfg}")
    for k, v in over.items():
        setattr(s, k, v)
    return s


WINDOWS = {  # (wy, wx, sy, sx)
    0: (5, 11, 1, 1),
    1: (5, 11, 3, 6),
    2: (5, 11, 3, 6),
    3: (5, 11, 1, 1),
    4: (5, 11, 1, 1),
}


def ministack_slices(n_dates: int, m: int) -> list[slice]:
    return [slice(i, min(n_dates, i + m)) for i in range(0, n_dates, m)]


def wrap(x):
    """Wrap angles to (-pi, pi]."""
    return torch.remainder(x + math.pi, 2 * math.pi) - math.pi
