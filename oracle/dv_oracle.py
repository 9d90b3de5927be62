"""FP64 CPU oracle of distributed shift-variant deblurring by Douglas-Rachford
consensus ("Distributed Deblurring of Large Images of Wide Field-Of-View").

TEST INFRASTRUCTURE ONLY.  The test suite, the package smoke check and the
CPU-baseline leg of the benchmark are its only callers.  The CUDA library and
its Python binding never import it and share no code with it; the two meet only
in the seeded input generators, which hold none of the method's arithmetic.

Everything is plain numpy in float64, written from the paper's statement of the
method, step by step, with no blocking, fusion or reordering beyond skipping
terms that are exactly zero:

  shift-variant blur by PSF interpolation ........ Sec. II-B
  non-circulant local blur, "valid" crop ......... Sec. II-B, Eq. (2)
  local cost f_i, consensus set .................. Sec. III-A, Eq. (4)
  D-R splitting, consensus prox .................. Sec. III-B, Lemma 1
  explicit per-pixel D-R updates ................. Sec. III-B
  alpha_i = gamma * omega_i ...................... Sec. III-B
  Distributed-Solver / Local-Solver .............. Algorithm 1
  Huber prior on forward differences ............. Sec. IV-A
  rho = 1, warm-started local solves ............. Sec. IV-B

Conventions.  Images are 2-D arrays indexed [row, col].  The observed image y
has shape (hy, wy); the unknown x has shape (hy + K - 1, wy + K - 1): H is the
rectangular "valid" operator of Eq. (2) (the sensor records a little less than
the optics see).  PSFs form an array (Gr, Gc, K, K) with K odd; convolution is
centred at (K // 2, K // 2), so y pixel (i, j) sits over x pixel
(i + K//2, j + K//2).  Interpolation weights are per-axis profiles wr (Gr, nxr)
and wc (Gc, nxc); grid PSF (a, b) has weight wr[a, R] * wc[b, C] at x pixel
(R, C).

Readings taken where the paper is silent, ambiguous or garbled:
 R1  Huber prior: applied per pixel to the Euclidean length of the
     forward-difference gradient (isotropic form), not to the whole vector.
 R2  Difference operator: forward differences, set to zero on the last row and
     column of each tile (Neumann); the paper's "circular" wrap-around would
     couple opposite tile edges.
 R3  PSF grid: G points per axis at c_a = a (n - 1)/(G - 1) in x-pixel
     coordinates, corners included; each weight is a tent of half-width
     (n - 1)/(G - 1); with G = 1 the single weight is 1 everywhere.
 R4  Consensus weights omega_i: separable trapezoids, 1 where no other tile
     reaches and at the outer border, ramping across each band shared by two
     neighbouring tiles with values (j + 1/2)/B (never 0, so the metric V stays
     positive definite), then divided by their sum over tiles, so that
     sum_i omega_i = 1 at every pixel.
 R5  Local-Solver: projected gradient on
     Phi_i(w) = f_i(w) + 1/2 ||w - u_i||^2_{alpha_i}, with step
     tau_i = 1 / (Wmax_i L_H + 8 lambda + gamma max omega_i) and
     L_H = (max_p sum_k |h_p(k)|) (sum_k max_p |h_p(k)|) >= ||H||^2
     (the paper runs VMLM-B; any convergent local solver is allowed).
     n_inner steps, warm-started from the current x_i.
 R6  Start: x_i = u_i = C_i x0, with x0 the observed image edge-replicated by
     K // 2 on every side unless x0 is given.
 R7  Output: x_hat = sum_i omega_i x_i / sum_i omega_i (Algorithm 1 returns the
     x_i only).
 R8  Fixed outer iteration count; the local solve at outer iteration k runs
     n_inner + k * inner_increment steps.
 R9  The consensus step uses the Lemma's normalised weighted mean, which equals
     Algorithm 1's unnormalised sum whenever sum_i omega_i = 1.
 R10 Noise weights W: 1 for uniform Gaussian noise, so lambda is relative to
     the unweighted data term; a per-pixel W (0 for unmeasured pixels) may be
     given.
 R19 Evaluation measures (Sec. IV-C names SNR and SSIM, citing Wang et al.
     2004, without formulas): SNR = 10 log10(||ref||^2 / ||x - ref||^2) dB over
     all pixels; SSIM as Wang et al. define it, averaged over every 11 x 11
     window inside the image (unit-sum Gaussian window of standard deviation
     1.5, C1 = (0.01 L)^2, C2 = (0.03 L)^2, L the dynamic range).
 R20 VMLM-B Local-Solver (local_solver="vmlmb"; the paper's solver, Sec. IV-B,
     whose steps the paper does not spell out): per tile, a limited-memory
     variable metric on Phi_i with m pairs, emptied at every local solve.
     Free set F = {w > 0 or g < 0}; two-loop recursion on the gradient
     restricted to F with full-vector pair products and H0 = (s'y / y'y) I of
     the newest pair; the direction is zeroed outside F.  With no pairs, or
     when g'd >= 0 (memory emptied), d = -tau_i (g on F): the projected-gradient
     step.  Armijo along w(a) = max(0, w + a d): Phi(w(a)) <= Phi(w) +
     1e-4 g'(w(a) - w), a = 1, 1/2, ..., at most 20 trials; no acceptance: stay
     and empty the memory.  The pair (s, y) is kept if s'y > 0 (the oldest of
     m + 1 dropped), else the memory is emptied.
 R21 VMLM-B stop at the objective's resolution (the paper runs a fixed
     number of VMLM-B iterations per local solve, Sec. IV-B): with stop_rel >
     0 a tile ends its local solve -- keeps its iterate for the remaining
     iterations -- as soon as the first-order decrease promised by a full step
     along its direction, -g'd, is at most stop_rel * |Phi_i(w)|.  Objectives
     formed from FP32 residuals do not resolve smaller changes (about 1e-7
     relative), so without the stop their Armijo tests fail on rounding alone.
     stop_rel = 0 (the default here) runs every iteration.
 R18 One PSF per block (weights="per_tile", the paper's own layout, Sec.
     III-A and III-C): the PSF grid is the tile grid and tile (tr, tc) blurs
     with PSF (tr, tc) alone, weight 1 on the whole tile; its step uses L_H of
     that PSF alone.  Blocks: G equal cells per axis of the x grid, x-tile i
     spanning cells i - 1 .. i + 1 (clipped to the image), the y-block being the
     x-tile less K - 1 rows (columns) at its end.  Neighbours share one cell,
     half an interior block, and with R4 the consensus weights become the
     first-order interpolation tents of the paper.

Pins: every function here is checked by the "not gpu" tests against closed
forms, library routines on special cases, invariants or brute force; none is
"parity unpinned".
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# First-order interpolation weights (Sec. II-B, Fig. 1), reading R3
# ---------------------------------------------------------------------------


def grid_spacing(n: int, G: int) -> float:
    """Distance between neighbouring PSF grid points along an axis of n pixels."""
    if G < 1:
        raise ValueError("G must be >= 1")
    return float("inf") if G == 1 else (n - 1) / (G - 1)


def bilinear_weights(n: int, G: int) -> np.ndarray:
    """Per-axis interpolation profiles, shape (G, n): tent of grid point a at t."""
    if G == 1:
        return np.ones((1, n))
    delta = grid_spacing(n, G)
    t = np.arange(n, dtype=np.float64)
    c = np.arange(G, dtype=np.float64) * delta
    return np.maximum(0.0, 1.0 - np.abs(t[None, :] - c[:, None]) / delta)


# ---------------------------------------------------------------------------
# Shift-variant blur H x = sum_p h_p * (w_p . x), valid part (Sec. II-B)
# ---------------------------------------------------------------------------


def _support(profile: np.ndarray):
    nz = np.nonzero(profile)[0]
    return (int(nz[0]), int(nz[-1]) + 1) if nz.size else None


def apply_H(x: np.ndarray, psfs: np.ndarray, wr: np.ndarray, wc: np.ndarray) -> np.ndarray:
    """y(i, j) = sum_p sum_k h_p(k) (w_p . x)(i + K-1 - k_r, j + K-1 - k_c).

    Each grid PSF blurs its weighted copy of x; the sum is restricted to the
    outputs whose K x K window meets the weight's support (the others receive
    exact zeros)."""
    Gr, Gc, K, _ = psfs.shape
    nxr, nxc = x.shape
    ny, nx = nxr - K + 1, nxc - K + 1
    y = np.zeros((ny, nx))
    for a in range(Gr):
        sr = _support(wr[a])
        if sr is None:
            continue
        for b in range(Gc):
            sc = _support(wc[b])
            if sc is None:
                continue
            s = np.outer(wr[a], wc[b]) * x
            i0, i1 = max(0, sr[0] - (K - 1)), min(ny, sr[1])
            j0, j1 = max(0, sc[0] - (K - 1)), min(nx, sc[1])
            if i0 >= i1 or j0 >= j1:
                continue
            h = psfs[a, b]
            for ka in range(K):
                for kb in range(K):
                    if h[ka, kb] == 0.0:
                        continue
                    y[i0:i1, j0:j1] += h[ka, kb] * s[i0 + K - 1 - ka:i1 + K - 1 - ka,
                                                     j0 + K - 1 - kb:j1 + K - 1 - kb]
    return y


def apply_Ht(r: np.ndarray, psfs: np.ndarray, wr: np.ndarray, wc: np.ndarray) -> np.ndarray:
    """g = H^T r: g(R, C) = sum_p w_p(R, C) sum_k h_p(k) r(R - (K-1) + k_r, C - (K-1) + k_c),
    r taken as zero outside its extent (the transpose of apply_H)."""
    Gr, Gc, K, _ = psfs.shape
    ny, nx = r.shape
    nxr, nxc = ny + K - 1, nx + K - 1
    rp = np.zeros((ny + 2 * (K - 1), nx + 2 * (K - 1)))
    rp[K - 1:K - 1 + ny, K - 1:K - 1 + nx] = r
    g = np.zeros((nxr, nxc))
    for a in range(Gr):
        sr = _support(wr[a])
        if sr is None:
            continue
        for b in range(Gc):
            sc = _support(wc[b])
            if sc is None:
                continue
            (R0, R1), (C0, C1) = sr, sc
            h = psfs[a, b]
            t = np.zeros((R1 - R0, C1 - C0))
            for ka in range(K):
                for kb in range(K):
                    if h[ka, kb] == 0.0:
                        continue
                    t += h[ka, kb] * rp[R0 + ka:R1 + ka, C0 + kb:C1 + kb]
            g[R0:R1, C0:C1] += np.outer(wr[a, R0:R1], wc[b, C0:C1]) * t
    return g


def apply_H_at(x, psfs, wr, wc, pts) -> np.ndarray:
    """(H x) at the listed output pixels, each summed on its own K x K window."""
    Gr, Gc, K, _ = psfs.shape
    out = np.empty(len(pts))
    for n, (i, j) in enumerate(pts):
        win = x[i:i + K, j:j + K]
        acc = 0.0
        for a in range(Gr):
            wra = wr[a, i:i + K]
            if not wra.any():
                continue
            for b in range(Gc):
                wcb = wc[b, j:j + K]
                if not wcb.any():
                    continue
                acc += np.sum(psfs[a, b, ::-1, ::-1] * np.outer(wra, wcb) * win)
        out[n] = acc
    return out


def apply_Ht_at(r, psfs, wr, wc, pts) -> np.ndarray:
    """(H^T r) at the listed x pixels, each summed on its own K x K window of r."""
    Gr, Gc, K, _ = psfs.shape
    ny, nx = r.shape
    rp = np.zeros((ny + 2 * (K - 1), nx + 2 * (K - 1)))
    rp[K - 1:K - 1 + ny, K - 1:K - 1 + nx] = r
    out = np.empty(len(pts))
    for n, (R, C) in enumerate(pts):
        win = rp[R:R + K, C:C + K]
        acc = 0.0
        for a in range(Gr):
            for b in range(Gc):
                w = wr[a, R] * wc[b, C]
                if w != 0.0:
                    acc += w * np.sum(psfs[a, b] * win)
        out[n] = acc
    return out


def lipschitz_bound_H(psfs: np.ndarray) -> float:
    """||H||^2 <= ||H||_1 ||H||_inf <= (max_p sum_k |h_p|)(sum_k max_p |h_p(k)|),
    using sum_p w_p <= 1 and w_p >= 0 (reading R5)."""
    a = np.abs(psfs.reshape(-1, psfs.shape[2] * psfs.shape[3]))
    return float(a.sum(axis=1).max() * a.max(axis=0).sum())


# ---------------------------------------------------------------------------
# Huber prior on forward differences (Sec. IV-A), readings R1 and R2
# ---------------------------------------------------------------------------


def forward_differences(x: np.ndarray):
    dr = np.zeros_like(x)
    dr[:-1, :] = x[1:, :] - x[:-1, :]
    dc = np.zeros_like(x)
    dc[:, :-1] = x[:, 1:] - x[:, :-1]
    return dr, dc


def huber_value(x: np.ndarray, delta: float) -> float:
    """phi(D x) = sum_l hub(|grad x(l)|), hub(s) = s^2/2 if s <= delta else delta (s - delta/2)."""
    dr, dc = forward_differences(x)
    s = np.sqrt(dr * dr + dc * dc)
    return float(np.sum(np.where(s <= delta, 0.5 * s * s, delta * (s - 0.5 * delta))))


def huber_gradient(x: np.ndarray, delta: float) -> np.ndarray:
    """D^T psi(D x) with psi(g) = g if |g| <= delta else delta g / |g|."""
    dr, dc = forward_differences(x)
    s = np.sqrt(dr * dr + dc * dc)
    kappa = np.where(s <= delta, 1.0, delta / np.where(s > 0.0, s, 1.0))
    pr, pc = kappa * dr, kappa * dc
    g = -pr - pc
    g[1:, :] += pr[:-1, :]
    g[:, 1:] += pc[:, :-1]
    return g


# ---------------------------------------------------------------------------
# Tiling, consensus weights, metric (Sec. III-A/C, Fig. 1), reading R4
# ---------------------------------------------------------------------------


def uniform_blocks(n: int, count: int, overlap: int):
    """[start, end) of `count` equal y-blocks covering n pixels, neighbours
    sharing about `overlap` pixels (start i = round(i (n - B)/(count - 1)))."""
    if count == 1:
        return [(0, n)]
    B = -(-(n + (count - 1) * overlap) // count)
    B = min(B, n)
    return [((i * (n - B) + (count - 1) // 2) // (count - 1),
             (i * (n - B) + (count - 1) // 2) // (count - 1) + B) for i in range(count)]


def consensus_profiles(xranges):
    """Per-tile 1-D profiles omega along one axis for x-ranges [s_i, e_i)."""
    t = [np.ones(e - s) for (s, e) in xranges]
    for i in range(len(xranges) - 1):
        s_i = xranges[i][0]
        s_n, e_i = xranges[i + 1][0], xranges[i][1]
        B = e_i - s_n
        if B <= 0:
            continue
        up = (np.arange(B) + 0.5) / B
        t[i + 1][:B] *= up
        t[i][s_n - s_i:] *= 1.0 - up
    n = max(e for _, e in xranges)
    total = np.zeros(n)
    for (s, e), ti in zip(xranges, t):
        total[s:e] += ti
    return [ti / total[s:e] for (s, e), ti in zip(xranges, t)]


@dataclass
class Layout:
    """Tile layout: y-blocks per tile row/column, x-tiles = y-blocks + K - 1."""
    hy: int
    wy: int
    K: int
    yrows: list
    ycols: list
    xrows: list = field(init=False)
    xcols: list = field(init=False)
    omega_r: list = field(init=False)
    omega_c: list = field(init=False)

    def __post_init__(self):
        K = self.K
        self.xrows = [(a, b + K - 1) for a, b in self.yrows]
        self.xcols = [(a, b + K - 1) for a, b in self.ycols]
        self.omega_r = consensus_profiles(self.xrows)
        self.omega_c = consensus_profiles(self.xcols)

    @property
    def tiles(self):
        return [(tr, tc) for tr in range(len(self.yrows)) for tc in range(len(self.ycols))]

    @property
    def nx(self):
        return self.hy + self.K - 1, self.wy + self.K - 1

    def xslice(self, tr, tc):
        (r0, r1), (c0, c1) = self.xrows[tr], self.xcols[tc]
        return slice(r0, r1), slice(c0, c1)

    def yslice(self, tr, tc):
        (r0, r1), (c0, c1) = self.yrows[tr], self.ycols[tc]
        return slice(r0, r1), slice(c0, c1)

    def omega(self, tr, tc):
        return np.outer(self.omega_r[tr], self.omega_c[tc])


def make_layout(hy, wy, K, n_tr, n_tc, overlap, yrows=None, ycols=None) -> Layout:
    yrows = yrows if yrows is not None else uniform_blocks(hy, n_tr, overlap)
    ycols = ycols if ycols is not None else uniform_blocks(wy, n_tc, overlap)
    return Layout(hy, wy, K, list(map(tuple, yrows)), list(map(tuple, ycols)))


def paper_blocks(ny: int, K: int, G: int):
    """[start, end) y-blocks of reading R18 on one axis: x-tile i covers cells
    i - 1 .. i + 1 of G equal cells of the n = ny + K - 1 x coordinates."""
    n = ny + K - 1
    cell = n / G
    out = []
    for i in range(G):
        x0 = 0 if i == 0 else int(np.floor((i - 0.5) * cell + 1e-9))
        x1 = n if i == G - 1 else int(np.floor((i + 1.5) * cell + 1e-9))
        out.append((x0, x1 - (K - 1)))
    return out


def paper_layout(hy, wy, K, Gr, Gc) -> "Layout":
    """Tile layout of reading R18 (one block per PSF grid point)."""
    return Layout(hy, wy, K, paper_blocks(hy, K, Gr), paper_blocks(wy, K, Gc))


def tile_operator(layout: "Layout", tr, tc, psfs, weights):
    """(PSFs, row weights, column weights) of tile (tr, tc)'s operator H_i:
    the interpolated operator restricted to the tile, or with
    weights == "per_tile" its own PSF alone with weight 1 (reading R18)."""
    if isinstance(weights, str):
        assert weights == "per_tile"
        (r0, r1), (c0, c1) = layout.xrows[tr], layout.xcols[tc]
        return psfs[tr:tr + 1, tc:tc + 1], np.ones((1, r1 - r0)), np.ones((1, c1 - c0))
    wr, wc = weights
    return (psfs,) + tile_weights(layout, tr, tc, wr, wc)


def tile_step(layout: Layout, tr, tc, psfs, W, lam, gamma) -> float:
    """tau_i of reading R5 (1 / Lipschitz bound of grad Phi_i); psfs are the
    PSFs of the tile's operator."""
    Wmax = 1.0 if W is None else float(np.max(W[layout.yslice(tr, tc)]))
    omax = float(layout.omega_r[tr].max() * layout.omega_c[tc].max())
    return 1.0 / (Wmax * lipschitz_bound_H(psfs) + 8.0 * lam + gamma * omax)


# ---------------------------------------------------------------------------
# Local-Solver: projected gradient on the prox objective (Algorithm 1), R5
# ---------------------------------------------------------------------------


def prox_objective(w, u, y_i, W_i, psfs, wr_i, wc_i, alpha_i, lam, delta) -> float:
    """Phi_i(w) = 1/2 ||y_i - H_i w||^2_W + lam phi(D w) + 1/2 ||w - u||^2_alpha (w >= 0)."""
    r = apply_H(w, psfs, wr_i, wc_i) - y_i
    data = 0.5 * np.sum((1.0 if W_i is None else W_i) * r * r)
    return float(data + lam * huber_value(w, delta) + 0.5 * np.sum(alpha_i * (w - u) ** 2))


def local_solve(w, u, y_i, W_i, psfs, wr_i, wc_i, alpha_i, lam, delta, tau, n_inner):
    """n_inner projected-gradient steps from w:
    r = W (H_i w - y_i); g = H_i^T r; grad = g + lam D^T psi(D w) + alpha (w - u);
    w <- max(0, w - tau grad)."""
    for _ in range(n_inner):
        r = apply_H(w, psfs, wr_i, wc_i) - y_i
        if W_i is not None:
            r = W_i * r
        g = apply_Ht(r, psfs, wr_i, wc_i)
        grad = g + lam * huber_gradient(w, delta) + alpha_i * (w - u)
        w = np.maximum(0.0, w - tau * grad)
    return w


def local_solve_vmlmb(w, u, y_i, W_i, psfs, wr_i, wc_i, alpha_i, lam, delta, tau, n_iter, m=5,
                      stop_rel=0.0, stats=None):
    """n_iter VMLM-B iterations of reading R20 on Phi_i from w, ending early
    under reading R21 when stop_rel > 0.  stats (a dict, optional) receives
    "trials" (Armijo trials of every iteration run) and "stopped_at" (the
    iteration at which the stop of R21 ended the solve, or None)."""
    def phi(v):
        return prox_objective(v, u, y_i, W_i, psfs, wr_i, wc_i, alpha_i, lam, delta)

    def grad(v):
        r = apply_H(v, psfs, wr_i, wc_i) - y_i
        if W_i is not None:
            r = W_i * r
        return apply_Ht(r, psfs, wr_i, wc_i) + lam * huber_gradient(v, delta) + alpha_i * (v - u)

    pairs = []            # (s, y, 1 / s'y), oldest first
    h0 = 1.0
    if stats is not None:
        stats.setdefault("trials", [])
        stats["stopped_at"] = None
    f, g = phi(w), grad(w)
    for it in range(n_iter):
        free = (w > 0) | (g < 0)
        q = np.where(free, g, 0.0)
        a = []
        for s, y, rho in reversed(pairs):
            ai = rho * float(np.sum(s * q))
            q = q - ai * y
            a.append(ai)
        if pairs:
            q = h0 * q
        for (s, y, rho), ai in zip(pairs, reversed(a)):
            b = rho * float(np.sum(y * q))
            q = q + (ai - b) * s
        d = np.where(free, -(1.0 if pairs else tau) * q, 0.0)
        if not float(np.sum(g * d)) < 0.0:
            pairs = []
            d = np.where(free, -tau * g, 0.0)
        if stop_rel > 0.0 and -float(np.sum(g * d)) <= stop_rel * abs(f):
            if stats is not None:
                stats["stopped_at"] = it
            break
        step, wt, ft = 1.0, None, None
        for trial in range(20):
            cand = np.maximum(0.0, w + step * d)
            fc = phi(cand)
            if fc <= f + 1e-4 * float(np.sum(g * (cand - w))):
                wt, ft = cand, fc
                break
            step *= 0.5
        if stats is not None:
            stats["trials"].append(trial + 1)
        if wt is None:
            pairs = []
            wt, ft = w.copy(), f
        gt = grad(wt)
        s, y = wt - w, gt - g
        sy, yy = float(np.sum(s * y)), float(np.sum(y * y))
        if sy > 0.0 and yy > 0.0:
            pairs = (pairs + [(s, y, 1.0 / sy)])[-m:]
            h0 = sy / yy
        else:
            pairs = []
        w, g, f = wt, gt, ft
    return w


# ---------------------------------------------------------------------------
# Consensus prox (Lemma 1) and dual update (Sec. III-B)
# ---------------------------------------------------------------------------


def consensus_average(layout: Layout, vs, alphas) -> np.ndarray:
    """z(l) = sum_{i in P_l^-} alpha_i(l) v_i(l) / sum_{i in P_l^-} alpha_i(l)."""
    num = np.zeros(layout.nx)
    den = np.zeros(layout.nx)
    for n, (tr, tc) in enumerate(layout.tiles):
        sl = layout.xslice(tr, tc)
        num[sl] += alphas[n] * vs[n]
        den[sl] += alphas[n]
    return num / den


def assemble(layout: Layout, xs) -> np.ndarray:
    """x_hat = sum_i omega_i x_i / sum_i omega_i (reading R7)."""
    return consensus_average(layout, xs, [layout.omega(tr, tc) for tr, tc in layout.tiles])


def start_image(y: np.ndarray, K: int) -> np.ndarray:
    """x0 of reading R6: y edge-replicated by K // 2 on every side."""
    return np.pad(y, K // 2, mode="edge")


def tile_weights(layout: Layout, tr, tc, wr, wc):
    (r0, r1), (c0, c1) = layout.xrows[tr], layout.xcols[tc]
    return wr[:, r0:r1], wc[:, c0:c1]


def objective(xhat, y, psfs, layout: Layout, lam, delta, W=None, weights=None):
    """F = sum_i [1/2 ||y_i - H_i C_i x||^2_W + lam phi(D C_i x)] (Eq. (4) at a
    consensus point).  weights: (wr, wc) profiles, None (bilinear) or
    "per_tile" (reading R18).  Returns (F, data term, prior sum)."""
    if weights is None:
        weights = (bilinear_weights(layout.nx[0], psfs.shape[0]),
                   bilinear_weights(layout.nx[1], psfs.shape[1]))
    data = prior = 0.0
    for tr, tc in layout.tiles:
        xi = xhat[layout.xslice(tr, tc)]
        pi, wri, wci = tile_operator(layout, tr, tc, psfs, weights)
        ri = apply_H(xi, pi, wri, wci) - y[layout.yslice(tr, tc)]
        Wi = 1.0 if W is None else W[layout.yslice(tr, tc)]
        data += 0.5 * float(np.sum(Wi * ri * ri))
        prior += huber_value(xi, delta)
    return data + lam * prior, data, prior


@dataclass
class SolveInfo:
    taus: list
    primal: list = field(default_factory=list)
    dual: list = field(default_factory=list)
    objective: list = field(default_factory=list)
    xs: list = field(default_factory=list)
    us: list = field(default_factory=list)


def solve(y, psfs, layout: Layout, lam, delta, gamma, rho, n_outer, n_inner,
          inner_increment=0, W=None, x0=None, weights=None, history=False,
          local_solver="pg", vm_memory=5, vm_stop_rel=0.0, vm_stats=None):
    """Algorithm 1 with the explicit D-R updates of Sec. III-B:
      x_i   <- Local-Solver(u_i; alpha_i, f_i)                    (all tiles)
      zbar  <- sum alpha_i (2 x_i - u_i) / sum alpha_i             (Lemma 1)
      u_i   <- u_i + rho (zbar - x_i)
    repeated n_outer times.  weights: (wr, wc) profiles, None (bilinear) or
    "per_tile" (reading R18).  Returns (x_hat, SolveInfo)."""
    assert local_solver in ("pg", "vmlmb"), local_solver
    K = psfs.shape[2]
    nxr, nxc = layout.nx
    if weights is None:
        weights = (bilinear_weights(nxr, psfs.shape[0]), bilinear_weights(nxc, psfs.shape[1]))
    ops = [tile_operator(layout, tr, tc, psfs, weights) for tr, tc in layout.tiles]
    x0 = start_image(y, K) if x0 is None else np.asarray(x0, dtype=np.float64)
    tiles = layout.tiles
    xs = [x0[layout.xslice(tr, tc)].copy() for tr, tc in tiles]
    us = [x.copy() for x in xs]
    alphas = [gamma * layout.omega(tr, tc) for tr, tc in tiles]
    taus = [tile_step(layout, tr, tc, op[0], W, lam, gamma) for op, (tr, tc) in zip(ops, tiles)]
    info = SolveInfo(taus=taus)
    zprev = x0
    for k in range(n_outer):
        ni = n_inner + k * inner_increment
        for n, (tr, tc) in enumerate(tiles):
            pi, wri, wci = ops[n]
            Wi = None if W is None else W[layout.yslice(tr, tc)]
            solver = local_solve if local_solver == "pg" else local_solve_vmlmb
            extra = ({} if local_solver == "pg" else
                     {"m": vm_memory, "stop_rel": vm_stop_rel, "stats": vm_stats})
            xs[n] = solver(xs[n], us[n], y[layout.yslice(tr, tc)], Wi, pi, wri, wci,
                           alphas[n], lam, delta, taus[n], ni, **extra)
        zbar = consensus_average(layout, [2.0 * x - u for x, u in zip(xs, us)], alphas)
        info.primal.append(float(np.sqrt(sum(np.sum((x - zbar[layout.xslice(tr, tc)]) ** 2)
                                             for x, (tr, tc) in zip(xs, tiles)))))
        info.dual.append(float(np.sqrt(np.sum((zbar - zprev) ** 2))))
        zprev = zbar
        us = [u + rho * (zbar[layout.xslice(tr, tc)] - x) for u, x, (tr, tc) in zip(us, xs, tiles)]
        if history:
            info.objective.append(objective(assemble(layout, xs), y, psfs, layout, lam, delta,
                                            W, weights)[0])
    info.xs, info.us = xs, us
    return assemble(layout, xs), info


# ---------------------------------------------------------------------------
# Evaluation measures (Sec. IV-C), reading R19
# ---------------------------------------------------------------------------


def snr_db(x: np.ndarray, ref: np.ndarray) -> float:
    """10 log10(||ref||^2 / ||x - ref||^2)."""
    x, ref = np.asarray(x, np.float64), np.asarray(ref, np.float64)
    err = float(np.sum((x - ref) ** 2))
    return float("inf") if err == 0.0 else 10.0 * np.log10(float(np.sum(ref * ref)) / err)


def ssim_window() -> np.ndarray:
    """11 x 11 circular Gaussian window, standard deviation 1.5, unit sum."""
    t = np.arange(11) - 5.0
    g = np.exp(-(t[:, None] ** 2 + t[None, :] ** 2) / (2 * 1.5 ** 2))
    return g / g.sum()


def ssim_map(x: np.ndarray, ref: np.ndarray, L: float = 1.0) -> np.ndarray:
    """SSIM of every 11 x 11 window inside the image (one value per window
    centre, shape (rows - 10, cols - 10)); local moments under ssim_window."""
    from scipy.signal import correlate2d
    x, ref = np.asarray(x, np.float64), np.asarray(ref, np.float64)
    w = ssim_window()
    mom = lambda a: correlate2d(a, w, mode="valid")
    mx, mr = mom(x), mom(ref)
    vx, vr, cxr = mom(x * x) - mx * mx, mom(ref * ref) - mr * mr, mom(x * ref) - mx * mr
    c1, c2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    return (2 * mx * mr + c1) * (2 * cxr + c2) / ((mx * mx + mr * mr + c1) * (vx + vr + c2))


def ssim(x: np.ndarray, ref: np.ndarray, L: float = 1.0) -> float:
    """Mean SSIM over the windows inside the image."""
    return float(np.mean(ssim_map(x, ref, L)))
