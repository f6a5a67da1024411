"""Seeded synthetic inputs for the TPFA single-phase pressure problem.

This module only draws numbers and lays out index sets; it contains none of
the finite-volume arithmetic (no transmissibility, no operator, no solver), so
both the CUDA path and the CPU oracle can consume what it produces.

Random numbers come from a counter-based generator so that any cell of any
grid can be drawn on its own, in O(1), without generating the rest of the
field (the full-size parity checks draw a few thousand sampled cells this way):

* SplitMix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom
  number generators", OOPSLA 2014) applied to ``key + (counter + 1) * GAMMA``;
  ``key`` mixes the seed and a stream id, ``counter`` is the draw index.
* Uniform on (0, 1): the top 53 bits, offset by half an ulp.
* Standard normal: Box-Muller (cos branch) on the uniforms of counters
  ``2*i`` and ``2*i + 1``.

Workload shapes follow the paper's structured 3D Cartesian mesh with X
innermost and Z outermost (Section IV): flat index ``i + nx*(j + ny*k)``.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = np.uint64(0xD1B54A32D192ED03)

# stream ids: one per kind of draw, so fields never share random numbers
STREAM_LNK = 1
STREAM_INSTANCE = 2
STREAM_CHANNEL = 3
STREAM_FIELD = 4


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64).copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        t = np.array([stream & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        return _mix(s * GAMMA + t * _STREAM_MUL)[0]


def bits(seed: int, stream: int, counter) -> np.ndarray:
    """64 random bits per counter value (counter-based SplitMix64)."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key(seed, stream) + (c + np.uint64(1)) * GAMMA)


def uniform(seed: int, stream: int, counter) -> np.ndarray:
    """Uniform doubles in (0, 1), one per counter."""
    b = bits(seed, stream, counter)
    return ((b >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def normal(seed: int, stream: int, draw) -> np.ndarray:
    """Standard normal doubles, one per draw index (Box-Muller, cos branch)."""
    d = np.asarray(draw, dtype=np.uint64)
    u1 = uniform(seed, stream, d * np.uint64(2))
    u2 = uniform(seed, stream, d * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ----------------------------------------------------------------------------
# permeability fields
# ----------------------------------------------------------------------------

def _draw_index(nx, ny, nz, cells, layer):
    cells = np.asarray(cells, dtype=np.int64)
    i = cells % nx
    j = (cells // nx) % ny
    k = cells // (nx * ny)
    return (i + nx * (j + ny * (k // layer))).astype(np.uint64)


def lognormal_at(nx, ny, nz, sigma, seed, cells, layer=1, stream=STREAM_LNK):
    """Permeability K = exp(sigma * N(0,1)) at the given flat cell indices.

    ``layer`` > 1 makes ln K constant over vertical runs of ``layer`` cells
    (one draw per (i, j, floor(k / layer))), the layered-correlation recipe of
    the paper-scale workload.
    """
    return np.exp(sigma * normal(seed, stream, _draw_index(nx, ny, nz, cells, layer)))


def lognormal_field(nx, ny, nz, sigma, seed, layer=1, stream=STREAM_LNK):
    """Whole permeability field (float64, length nx*ny*nz, X innermost)."""
    if layer == 1:
        draws = np.arange(nx * ny * nz, dtype=np.uint64)
        return np.exp(sigma * normal(seed, stream, draws))
    nzl = -(-nz // layer)
    base = np.exp(sigma * normal(seed, stream, np.arange(nx * ny * nzl, dtype=np.uint64)))
    base = base.reshape(nzl, ny * nx)
    out = np.repeat(base, layer, axis=0)[:nz]
    return np.ascontiguousarray(out).reshape(-1)


def channelized_field(nx, ny, nz, sigma, seed, n_channels=8, width=4, thickness=8,
                      amplitude=16.0, wavelength=128.0, contrast=1e4):
    """Lognormal background with sinusoidal high-permeability channels.

    Each channel is ``width`` cells wide in y and ``thickness`` layers thick in
    z, centred on y_c + amplitude*sin(2*pi*x/wavelength + phi); K inside is
    multiplied by ``contrast``.  Channel centre, layer and phase come from the
    seed.
    """
    K = lognormal_field(nx, ny, nz, sigma, seed).reshape(nz, ny, nx)
    return np.where(channel_mask(nx, ny, nz, seed, n_channels, width, thickness, amplitude,
                                 wavelength), K * contrast, K).reshape(-1)


def channel_mask(nx, ny, nz, seed, n_channels=8, width=4, thickness=8, amplitude=16.0,
                 wavelength=128.0):
    """Cells inside any of the sinusoidal channels (bool, shape (nz, ny, nx))."""
    inside_any = np.zeros((nz, ny, nx), dtype=bool)
    u = uniform(seed, STREAM_CHANNEL, np.arange(3 * n_channels, dtype=np.uint64)).reshape(n_channels, 3)
    x = np.arange(nx, dtype=np.float64)
    jj = np.arange(ny)[:, None]
    for c in range(n_channels):
        yc = u[c, 0] * ny
        z0 = int(u[c, 1] * max(nz - thickness, 1))
        phi = 2.0 * np.pi * u[c, 2]
        centre = yc + amplitude * np.sin(2.0 * np.pi * x / wavelength + phi)  # per x
        inside = np.abs(jj - centre[None, :]) < 0.5 * width                  # (ny, nx)
        inside_any[z0:z0 + thickness] |= inside[None, :, :]
    return inside_any


# ----------------------------------------------------------------------------
# boundary and source index sets
# ----------------------------------------------------------------------------

def dirichlet_faces(nx, ny, nz, axis="x", p_hi=1.0, p_lo=0.0):
    """Dirichlet cells on the two end layers of one axis.

    Returns (mask uint8[N], pD float64[N]): mask=1 on the layer index 0 and
    the last layer of ``axis``; pD = p_hi on the first, p_lo on the last.
    """
    mask = np.zeros((nz, ny, nx), dtype=np.uint8)
    pD = np.zeros((nz, ny, nx), dtype=np.float64)
    if axis == "x":
        mask[:, :, 0] = 1; mask[:, :, -1] = 1
        pD[:, :, 0] = p_hi; pD[:, :, -1] = p_lo
    elif axis == "y":
        mask[:, 0, :] = 1; mask[:, -1, :] = 1
        pD[:, 0, :] = p_hi; pD[:, -1, :] = p_lo
    elif axis == "z":
        mask[0] = 1; mask[-1] = 1
        pD[0] = p_hi; pD[-1] = p_lo
    else:
        raise ValueError(axis)
    return mask.reshape(-1), pD.reshape(-1)


def well_pair(nx, ny, nz, rate=1.0):
    """Injector +rate at cell (0,0,0) and producer -rate at the opposite corner."""
    idx = np.array([0, (nx - 1) + nx * ((ny - 1) + ny * (nz - 1))], dtype=np.int64)
    val = np.array([rate, -rate], dtype=np.float64)
    return idx, val


def dense_sources(n_cells, idx, val):
    q = np.zeros(n_cells, dtype=np.float64)
    np.add.at(q, idx, val)
    return q


def smooth_field(nx, ny, nz, seed, modes=4):
    """A smooth random field (sum of a few low-frequency cosines), float64."""
    u = uniform(seed, STREAM_FIELD, np.arange(4 * modes, dtype=np.uint64)).reshape(modes, 4)
    i = np.arange(nx)[None, None, :] / max(nx, 1)
    j = np.arange(ny)[None, :, None] / max(ny, 1)
    k = np.arange(nz)[:, None, None] / max(nz, 1)
    f = np.zeros((nz, ny, nx))
    for m in range(modes):
        f += np.cos(2 * np.pi * ((m % 3 + 1) * u[m, 0] * i + (m % 2 + 1) * u[m, 1] * j
                                 + u[m, 2] * k) + 2 * np.pi * u[m, 3])
    return f.reshape(-1) / modes


def uniform_field(n, seed, lo=-1.0, hi=1.0, stream=STREAM_FIELD):
    return lo + (hi - lo) * uniform(seed, stream, np.arange(n, dtype=np.uint64))


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def small_dirichlet(seed=0, n=32, sigma=1.0):
    """32^3 grid, i.i.d. ln K ~ N(0, sigma^2), p=1 / p=0 on the x end layers."""
    nx = ny = nz = n
    K = lognormal_field(nx, ny, nz, sigma, seed)
    mask, pD = dirichlet_faces(nx, ny, nz, "x", 1.0, 0.0)
    return dict(nx=nx, ny=ny, nz=nz, K=K, mask=mask, pD=pD, d=0.0,
                src_idx=np.zeros(0, np.int64), src_val=np.zeros(0))


def channelized(seed=0, n=256, sigma=2.0, contrast=1e4):
    """Mixed-precision workload: n^3 lognormal background (sigma) with eight
    sinusoidal channels 4 cells wide, 8 layers thick, `contrast` times more
    permeable; p = 1 / 0 on the x end layers."""
    K = channelized_field(n, n, n, sigma, seed, contrast=contrast)
    mask, pD = dirichlet_faces(n, n, n, "x", 1.0, 0.0)
    return dict(nx=n, ny=n, nz=n, K=K, mask=mask, pD=pD, d=0.0,
                src_idx=np.zeros(0, np.int64), src_val=np.zeros(0))


ENSEMBLE_SIZES = ((48, 48, 24), (64, 64, 32), (96, 96, 48), (128, 128, 64))


def ensemble(seed=0, n_inst=96, sizes=ENSEMBLE_SIZES, sigma_range=(0.5, 2.5)):
    """Batched workload: n_inst realizations, each with a size drawn uniformly
    from `sizes`, ln K ~ N(0, sigma^2) with sigma ~ U(sigma_range), Dirichlet
    end layers on an axis drawn from {x, y, z} with p_hi ~ U(0.5, 2), p_lo = 0.
    Returns a list of per-instance dicts (the K seeds differ per instance)."""
    u = uniform(seed, STREAM_INSTANCE, np.arange(4 * n_inst, dtype=np.uint64)).reshape(n_inst, 4)
    out = []
    for i in range(n_inst):
        nx, ny, nz = sizes[min(int(u[i, 0] * len(sizes)), len(sizes) - 1)]
        sigma = sigma_range[0] + (sigma_range[1] - sigma_range[0]) * u[i, 1]
        axis = "xyz"[min(int(u[i, 2] * 3), 2)]
        p_hi = 0.5 + 1.5 * u[i, 3]
        K = lognormal_field(nx, ny, nz, sigma, seed * 1000003 + i + 1)
        mask, pD = dirichlet_faces(nx, ny, nz, axis, p_hi, 0.0)
        out.append(dict(nx=nx, ny=ny, nz=nz, K=K, mask=mask, pD=pD, d=0.0, sigma=sigma,
                        axis=axis, p_hi=p_hi))
    return out


def paper_scale(seed=0, nx=1024, ny=1024, nz=256, sigma=1.5, layer=8, d=1e-3):
    """Layered lognormal field, accumulation diagonal d, corner well pair, no Dirichlet."""
    K = lognormal_field(nx, ny, nz, sigma, seed, layer=layer)
    idx, val = well_pair(nx, ny, nz)
    return dict(nx=nx, ny=ny, nz=nz, K=K, mask=None, pD=None, d=d,
                src_idx=idx, src_val=val)
