"""Kaiser-Bessel gridding NUFFT with density compensation (Sec. 2.1, Eq. 5).

Target (Eq. 1 with density compensation, A = W^1/2 F C):
    y_c[i] = sqrt(w_i) D^-1/2 sum_r c_c[r] x[r] exp(-i 2 pi <f_i, r>)
with r the centred integer voxel coordinates.  ``nudft_fwd`` evaluates this sum directly.

Gridding approximation (Beatty et al. 2005, cited for F~_n in Sec. 2.1), step by step:
  (i)   divide c_c x by the separable deapodisation psi(r) = prod_ax Phi(r_ax / G_ax), where
        Phi is the continuous Fourier transform of the KB kernel phi below, and by sqrt(D);
  (ii)  zero-pad to the oversampled grid G, centred;
  (iii) centred unnormalised DFT on the G grid;
  (iv)  interpolate: sum over the W^nd box of phi(g - j) * grid[j mod G] (box of binning.py);
  (v)   multiply by sqrt(w).
The adjoint is the exact conjugate transpose of (i)-(v).

Kernel (W = 4, oversampling alpha = 1.25):
    phi(u) = I0(beta sqrt(1 - (2u/W)^2)) / I0(beta) for |u| <= W/2, per axis,
    beta = pi sqrt((W/alpha)^2 (alpha - 1/2)^2 - 0.8)            (Beatty 2005),
    Phi(nu) = W sinh(sqrt(beta^2 - (pi W nu)^2)) / (sqrt(beta^2 - (pi W nu)^2) I0(beta)),
with sin in place of sinh past the zero.
"""
from __future__ import annotations

import numpy as np

from . import binning, fftlib

W = binning.KB_WIDTH


def kb_beta(width=W, alpha=1.25):
    return np.pi * np.sqrt((width / alpha) ** 2 * (alpha - 0.5) ** 2 - 0.8)


def kb_phi(u, beta, width=W):
    u = np.asarray(u, dtype=np.float64)
    arg = 1.0 - (2.0 * u / width) ** 2
    out = np.where(arg >= 0, np.i0(beta * np.sqrt(np.clip(arg, 0, None))) / np.i0(beta), 0.0)
    return out


def kb_phi_hat(nu, beta, width=W):
    nu = np.asarray(nu, dtype=np.float64)
    z2 = beta ** 2 - (np.pi * width * nu) ** 2
    z = np.sqrt(np.abs(z2))
    with np.errstate(invalid="ignore", divide="ignore"):
        val = np.where(z2 > 0, np.sinh(z) / np.where(z > 0, z, 1.0),
                       np.where(z > 0, np.sin(z) / np.where(z > 0, z, 1.0), 1.0))
    val = np.where(z == 0, 1.0, val)
    return width * val / np.i0(beta)


def deapod(img_shape, grid, beta):
    """psi(r) on the image grid (separable product), float64 [*img_shape]."""
    out = np.ones(img_shape)
    for ax, (n, G) in enumerate(zip(img_shape, grid)):
        r = np.arange(n) - n // 2
        v = kb_phi_hat(r / G, beta)
        shp = [1] * len(img_shape)
        shp[ax] = n
        out = out * v.reshape(shp)
    return out


def _cdft(u, axes, inverse):
    """Centred unnormalised DFT (inverse: its conjugate transpose) over ``axes``."""
    scale = np.sqrt(np.prod([u.shape[a] for a in axes]))
    sh = np.fft.ifftshift(u, axes=axes)
    t = fftlib.ifftn(sh, axes=axes, norm="ortho") if inverse else fftlib.fftn(sh, axes=axes, norm="ortho")
    return np.fft.fftshift(t, axes=axes) * scale


class Plan:
    """Discrete choices shared by the forward and adjoint gridding operators."""

    def __init__(self, traj, img_shape, grid, alpha=1.25):
        self.img = tuple(int(v) for v in img_shape)
        self.grid = tuple(int(v) for v in grid)
        self.nd = len(self.img)
        self.beta = kb_beta(W, alpha)
        self.g = binning.grid_coords(traj, self.grid).astype(np.float64)  # [N, nd]
        self.j0 = binning.kernel_box_start(self.g)                          # [N, nd]
        self.psi = deapod(self.img, self.grid, self.beta)
        self.D = int(np.prod(self.img))
        self.N = traj.shape[0]
        # per-axis weights [nd][N, W] and wrapped indices
        self.wts = []
        self.idx = []
        for ax in range(self.nd):
            js = self.j0[:, ax:ax + 1] + np.arange(W)[None, :]
            self.wts.append(kb_phi(self.g[:, ax:ax + 1] - js, self.beta))
            self.idx.append(np.mod(js, self.grid[ax]))
        self.pad = [(G - n) // 2 for n, G in zip(self.img, self.grid)]

    def _box_iter(self):
        import itertools
        for offs in itertools.product(range(W), repeat=self.nd):
            w = np.ones(self.N)
            flat = np.zeros(self.N, dtype=np.int64)
            for ax, o in enumerate(offs):
                w = w * self.wts[ax][:, o]
                flat = flat * self.grid[ax] + self.idx[ax][:, o]
            yield w, flat

    def interp(self, grid_vals):
        """Step (iv): y[i] = sum_box phi(g_i - j) grid[j mod G]."""
        gflat = grid_vals.reshape(-1)
        out = np.zeros(self.N, dtype=np.complex128)
        for w, flat in self._box_iter():
            out += w * gflat[flat]
        return out

    def spread(self, y):
        """Adjoint of interp: grid[j] = sum_i phi(g_i - j) y[i]."""
        G = int(np.prod(self.grid))
        re = np.zeros(G)
        im = np.zeros(G)
        for w, flat in self._box_iter():
            re += np.bincount(flat, weights=w * y.real, minlength=G)
            im += np.bincount(flat, weights=w * y.imag, minlength=G)
        return (re + 1j * im).reshape(self.grid)

    def pad_img(self, u):
        out = np.zeros(self.grid, dtype=np.complex128)
        sl = tuple(slice(p, p + n) for p, n in zip(self.pad, self.img))
        out[sl] = u
        return out

    def crop_img(self, g):
        sl = tuple(slice(p, p + n) for p, n in zip(self.pad, self.img))
        return g[sl]


def nufft_fwd(plan, u):
    """Single-coil gridding NUFFT of an image u (no maps, no dcf): steps (i)-(iv)."""
    v = u / plan.psi / np.sqrt(plan.D)
    gv = _cdft(plan.pad_img(v), tuple(range(plan.nd)), inverse=False)
    return plan.interp(gv)


def nufft_adj(plan, y):
    """Exact adjoint of nufft_fwd."""
    gv = plan.spread(y)
    v = _cdft(gv, tuple(range(plan.nd)), inverse=True)
    return plan.crop_img(v) / plan.psi / np.sqrt(plan.D)


def sense_fwd(plan, x, maps, dcf):
    """A x with A = W^1/2 F C (Eq. 5): y[c] = sqrt(w) * NUFFT(c_c * x).  Returns [C, N]."""
    sw = np.sqrt(np.asarray(dcf, dtype=np.float64))
    return np.stack([sw * nufft_fwd(plan, maps[c] * x) for c in range(maps.shape[0])])


def sense_adj(plan, y, maps, dcf):
    """A^H y = sum_c conj(c_c) * NUFFT^H(sqrt(w) * y_c)."""
    sw = np.sqrt(np.asarray(dcf, dtype=np.float64))
    out = np.zeros(plan.img, dtype=np.complex128)
    for c in range(maps.shape[0]):
        out += np.conj(maps[c]) * nufft_adj(plan, sw * y[c])
    return out


def nudft_fwd(x, maps, traj, dcf, chunk=4096):
    """Exact Eq. 1 (with sqrt(w)): direct O(N D) sum, for tiny inputs."""
    shape = x.shape
    D = int(np.prod(shape))
    r = np.stack(np.meshgrid(*[np.arange(n) - n // 2 for n in shape], indexing="ij"), -1).reshape(D, -1)
    f = np.asarray(traj, dtype=np.float64)
    sw = np.sqrt(np.asarray(dcf, dtype=np.float64))
    C = maps.shape[0]
    out = np.zeros((C, f.shape[0]), dtype=np.complex128)
    cx = (maps * x[None]).reshape(C, D)
    for s in range(0, f.shape[0], chunk):
        E = np.exp(-2j * np.pi * (f[s:s + chunk] @ r.T.astype(np.float64))) / np.sqrt(D)
        out[:, s:s + chunk] = (cx @ E.T) * sw[None, s:s + chunk]
    return out
