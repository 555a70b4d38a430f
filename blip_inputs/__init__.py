"""Seeded synthetic inputs for the periodic cubic-blip orbital evaluator.

This module is shared by the FP64 oracle, the tests and the benchmark, and it
holds none of the evaluator's arithmetic: no B-spline, no stencil, no
contraction.  It only makes the things an evaluation consumes:

* coefficient tables ``[n1][n2][n3][n_orb]`` (orbital index fastest), smooth
  random fields standing in for the precomputed orbital coefficients that the
  paper reads from an input file (Sec. II.B, after Eq. 7);
* electron positions: uniform in the cell, and walker configurations with
  Gaussian trial moves (the quasi-simultaneous batches of Sec. IV.A);
* ragged walker offsets.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
value(key, i) = mix(key + (i + 1) * 0x9E3779B97F4A7C15), where mix is the
SplitMix64 finaliser.  Uniform doubles take the top 53 bits; normals use the
Box-Muller transform on consecutive pairs.  Every draw is addressed by
(key, counter), so any subset of a large input can be regenerated exactly.

Table recipe (per orbital l): i.i.d. N(0, 1) values on the grid (complex: real
and imaginary parts each N(0, 1)), a forward FFT, multiplication of mode
m = (m1, m2, m3) (signed integer indices) by exp(-|m|^2 / (2 sigma^2)) with
sigma = 3 grid modes, an inverse FFT (real part for real tables), and a
rescale so that the orbital's coefficients have RMS 1.
"""
from __future__ import annotations

import concurrent.futures as _cf
import os
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, *tags: int) -> np.uint64:
    """Derive a 64-bit stream key from a seed and integer tags."""
    k = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for t in tags:
            k = _mix(np.uint64(k) + np.uint64(t & 0xFFFFFFFFFFFFFFFF) * _GAMMA
                     + np.uint64(0x632BE59BD9B4E019))
    return np.uint64(k)


def raw_u64(key: np.uint64, counters: np.ndarray) -> np.ndarray:
    """SplitMix64 outputs for stream ``key`` at the given counters."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(key) + (c + np.uint64(1)) * _GAMMA)


def uniform(key: np.uint64, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits."""
    return (raw_u64(key, counters) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(key: np.uint64, start: int, count: int) -> np.ndarray:
    """``count`` standard normals: Box-Muller on counter pairs (2k, 2k+1).

    Normal number ``start + i`` is the cosine (even) or sine (odd) branch of
    pair ``(start + i) // 2``, so a draw does not depend on how a range is cut.
    """
    if count <= 0:
        return np.zeros(0)
    p0 = start // 2
    p1 = (start + count + 1) // 2
    pairs = np.arange(p0, p1, dtype=np.uint64)
    u1 = ((raw_u64(key, 2 * pairs) >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u2 = (raw_u64(key, 2 * pairs + np.uint64(1)) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    out = np.empty(2 * len(pairs))
    out[0::2] = rad * np.cos(ang)
    out[1::2] = rad * np.sin(ang)
    off = start - 2 * p0
    return out[off:off + count]


# ---------------------------------------------------------------------------
# cells
# ---------------------------------------------------------------------------

def cubic_lattice(a: float) -> np.ndarray:
    """Row i = lattice vector a_i (bohr)."""
    return np.diag([a, a, a]).astype(np.float64)


def tetragonal_lattice(a: float, c: float) -> np.ndarray:
    return np.diag([a, a, c]).astype(np.float64)


# ---------------------------------------------------------------------------
# coefficient tables
# ---------------------------------------------------------------------------

def _smooth_chunk(grid, l0, l1, seed, sigma, is_complex):
    n1, n2, n3 = grid
    P = n1 * n2 * n3
    key = stream_key(seed, 0x7AB1E)
    per = 2 * P if is_complex else P
    noise = normal(key, l0 * per, (l1 - l0) * per).reshape(l1 - l0, per)
    m1 = np.fft.fftfreq(n1) * n1
    m2 = np.fft.fftfreq(n2) * n2
    if is_complex:
        field_ = (noise[:, :P] + 1j * noise[:, P:]).reshape(l1 - l0, n1, n2, n3)
        m3 = np.fft.fftfreq(n3) * n3
        filt = np.exp(-(m1[:, None, None] ** 2 + m2[None, :, None] ** 2
                        + m3[None, None, :] ** 2) / (2.0 * sigma * sigma))
        f = np.fft.fftn(field_, axes=(1, 2, 3)) * filt
        out = np.fft.ifftn(f, axes=(1, 2, 3))
        rms = np.sqrt(np.mean(np.abs(out) ** 2, axis=(1, 2, 3)))
    else:
        field_ = noise.reshape(l1 - l0, n1, n2, n3)
        m3 = np.fft.rfftfreq(n3) * n3
        filt = np.exp(-(m1[:, None, None] ** 2 + m2[None, :, None] ** 2
                        + m3[None, None, :] ** 2) / (2.0 * sigma * sigma))
        f = np.fft.rfftn(field_, axes=(1, 2, 3)) * filt
        out = np.fft.irfftn(f, s=(n1, n2, n3), axes=(1, 2, 3))
        rms = np.sqrt(np.mean(out * out, axis=(1, 2, 3)))
    out /= rms[:, None, None, None]
    return out


def smooth_random_table(grid, n_orb: int, seed: int = 0, sigma: float = 3.0,
                        is_complex: bool = False, dtype=None,
                        threads: int | None = None, orb_chunk: int = 16) -> np.ndarray:
    """Smooth random coefficient table, shape ``[n1][n2][n3][n_orb]``.

    Real tables are float64 (or ``dtype``); complex tables are complex128 (or
    ``dtype``).  Orbital ``l`` depends only on (seed, l), never on n_orb or
    on how the work is chunked.
    """
    grid = tuple(int(g) for g in grid)
    if dtype is None:
        dtype = np.complex128 if is_complex else np.float64
    out = np.empty(grid + (n_orb,), dtype=dtype)
    chunks = [(l0, min(n_orb, l0 + orb_chunk)) for l0 in range(0, n_orb, orb_chunk)]

    def work(c):
        l0, l1 = c
        blk = _smooth_chunk(grid, l0, l1, seed, sigma, is_complex)
        out[..., l0:l1] = np.moveaxis(blk, 0, -1)

    nt = threads or min(16, os.cpu_count() or 1)
    if nt <= 1 or len(chunks) == 1:
        for c in chunks:
            work(c)
    else:
        with _cf.ThreadPoolExecutor(nt) as ex:
            list(ex.map(work, chunks))
    return out


def spectral_table(grid, orbitals, seed: int = 0, sigma: float = 3.0, cutoff: int | None = None,
                   device="cpu", out=None, chunk: int = 8):
    """Smooth random COMPLEX table synthesised in Fourier space (torch).

    The same statistics as ``smooth_random_table(is_complex=True)`` with a
    cheaper recipe for large supercell grids: the DFT of complex white noise is
    itself i.i.d. complex Gaussian, so each orbital draws N(0, 1) real and
    imaginary parts for every mode m with |m_a| <= cutoff (default 5 sigma;
    the Gaussian filter is below 4e-6 beyond it), multiplies mode m by
    exp(-|m|^2 / (2 sigma^2)), inverse-FFTs on the full grid and rescales to
    coefficient RMS 1.  ``orbitals`` is a range (or count): orbital l depends
    only on (seed, l), so any subset of orbitals can be regenerated alone.
    Returns (or fills ``out``) a complex128 tensor [n1][n2][n3][len(orbitals)]
    on ``device``.
    """
    import torch
    if isinstance(orbitals, int):
        orbitals = range(orbitals)
    grid = tuple(int(g) for g in grid)
    K = int(cutoff if cutoff is not None else int(np.ceil(5 * sigma)))
    ks = [min(K, (n - 1) // 2) for n in grid]
    axes = [np.arange(-k, k + 1) for k in ks]
    box = tuple(len(a) for a in axes)
    M = int(np.prod(box))
    m2 = (axes[0][:, None, None] ** 2 + axes[1][None, :, None] ** 2
          + axes[2][None, None, :] ** 2).astype(np.float64)
    filt = torch.from_numpy(np.exp(-m2 / (2.0 * sigma * sigma))).to(device)
    idx = [torch.from_numpy(np.mod(a, n)).to(device) for a, n in zip(axes, grid)]
    L = len(orbitals)
    if out is None:
        out = torch.empty(grid + (L,), dtype=torch.complex128, device=device)
    key = stream_key(seed, 0x5BEC7)
    ol = list(orbitals)
    for c0 in range(0, L, chunk):
        ls = ol[c0:c0 + chunk]
        G = torch.zeros((len(ls),) + grid, dtype=torch.complex128, device=device)
        for j, l in enumerate(ls):
            z = torch.from_numpy(normal(key, 2 * M * l, 2 * M)).to(device)
            F = torch.complex(z[:M], z[M:]).reshape(box) * filt
            G[j][idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]] = F
        blk = torch.fft.ifftn(G, dim=(1, 2, 3))
        rms = torch.sqrt(torch.mean(blk.real ** 2 + blk.imag ** 2, dim=(1, 2, 3)))
        blk /= rms[:, None, None, None]
        out[..., c0:c0 + len(ls)] = blk.permute(1, 2, 3, 0)
        del G, blk
    return out


# ---------------------------------------------------------------------------
# positions
# ---------------------------------------------------------------------------

def uniform_positions(lattice: np.ndarray, n: int, seed: int, stream: int = 0) -> np.ndarray:
    """``n`` positions uniform in the cell spanned by the rows of ``lattice``."""
    key = stream_key(seed, 0x9051, stream)
    u = uniform(key, np.arange(3 * n, dtype=np.uint64)).reshape(n, 3)
    return u @ np.asarray(lattice, dtype=np.float64)


def walker_positions(lattice: np.ndarray, n_walkers: int, n_per_walker: int,
                     batch, seed: int, move_sigma: float = 0.3):
    """Trial moves of a batch of walkers (quasi-simultaneous batches).

    Walker w has a uniform base configuration of ``n_per_walker`` electrons
    (stream (seed, w)); its first ``batch[w]`` electrons receive a Gaussian
    trial move r' = r + N(0, move_sigma^2) per component.  Returns
    ``(positions [E][3], offsets [W+1] int32)`` with the walkers' moved
    electrons stored contiguously.
    """
    batch = np.broadcast_to(np.asarray(batch, dtype=np.int64), (n_walkers,))
    offs = np.zeros(n_walkers + 1, dtype=np.int64)
    offs[1:] = np.cumsum(batch)
    pos = np.empty((int(offs[-1]), 3))
    lat = np.asarray(lattice, dtype=np.float64)
    for w in range(n_walkers):
        b = int(batch[w])
        if b > n_per_walker:
            raise ValueError("batch larger than the walker")
        key = stream_key(seed, 0x3A1C, w)
        u = uniform(key, np.arange(3 * b, dtype=np.uint64)).reshape(b, 3)
        mkey = stream_key(seed, 0x30FE, w)
        d = normal(mkey, 0, 3 * b).reshape(b, 3) * move_sigma
        pos[offs[w]:offs[w + 1]] = u @ lat + d
    return pos, offs.astype(np.int32)


def ragged_batch_sizes(n_walkers: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Batch sizes uniform in {lo..hi}."""
    key = stream_key(seed, 0x5A66ED)
    u = uniform(key, np.arange(n_walkers, dtype=np.uint64))
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    """One synthetic workload: the cell, the grid, the orbital count and how
    positions are drawn."""
    name: str
    lattice: np.ndarray
    grid: tuple
    n_orb: int
    is_complex: bool = False
    table_seed: int = 0
    pos_seed: int = 0
    n_walkers: int = 1
    n_per_walker: int = 0
    batch: object = None        # int, array, or "ragged"
    ragged: tuple = None        # (lo, hi) for ragged batch sizes
    uniform_n: int = 0          # >0: plain uniform positions (single walker)
    extra: dict = field(default_factory=dict)
    pos_lattice: np.ndarray = None   # cell the positions are drawn in (None: lattice)

    def positions(self):
        """(positions [E][3] float64, offsets [W+1] int32)."""
        cell = self.lattice if self.pos_lattice is None else self.pos_lattice
        if self.uniform_n:
            p = uniform_positions(cell, self.uniform_n, self.pos_seed)
            return p, np.array([0, self.uniform_n], dtype=np.int32)
        if self.ragged is not None:
            b = ragged_batch_sizes(self.n_walkers, self.ragged[0], self.ragged[1], self.pos_seed)
        else:
            b = self.batch
        return walker_positions(cell, self.n_walkers, self.n_per_walker, b, self.pos_seed)

    def table(self, dtype=None, threads=None, device="cpu", orbitals=None):
        """The coefficient table.  Complex supercell workloads use the
        Fourier-space recipe (``spectral_table``, a torch tensor on
        ``device``); the others the grid-noise recipe (numpy, host)."""
        if self.extra.get("spectral"):
            return spectral_table(self.grid, orbitals if orbitals is not None else self.n_orb,
                                  self.table_seed, device=device)
        return smooth_random_table(self.grid, self.n_orb, self.table_seed,
                                   is_complex=self.is_complex, dtype=dtype, threads=threads)

    @property
    def table_rows(self):
        return self.grid[0] * self.grid[1] * self.grid[2]


TIO2_CELL = tetragonal_lattice(17.4, 11.2)
TIO2_GRID = (72, 72, 48)


def workload(name: str, **kw) -> Workload:
    """Named synthetic workloads.

    * ``cubic16``: cubic cell 10 bohr, 16^3 grid, 8 real orbitals, 64 uniform
      positions (seed 0).
    * ``tio2``: tetragonal 17.4 x 17.4 x 11.2 bohr, 72 x 72 x 48 grid, 768 real
      orbitals, 1,536 uniform positions (the 1,536-electron TiO2 solid of the
      paper's benchmark table).
    * ``tio2_batch``: the same table, 256 walkers, ``batch`` moved electrons
      per walker (keyword ``batch``, default 1536).
    * ``tio2_precision``: the same table, 1,024 walkers x 1,536 electrons.
    * ``tio2_kpoints``: the primitive cell of the TiO2 cell (4.35 x 4.35 x 2.8
      bohr, a quarter along each axis), 18 x 18 x 12 grid, 64 k-points (the
      4 x 4 x 4 mesh kappa in {0, 1/4, 1/2, 3/4}^3) x 6 complex orbitals =
      384 complex orbitals (a 15 MB complex64 table), positions of 256
      walkers x ``batch`` moves drawn in the 4 x 4 x 4 supercell (the TiO2
      cell); ``extra`` holds kfrac [64][3] and koffs [65].
    * ``tio2_super_complex``: 2 x 2 x 2 supercell (34.8 x 34.8 x 22.4 bohr),
      144 x 144 x 96 grid, 1,536 complex orbitals (Fourier-space table
      recipe), 512 walkers with batch sizes uniform in {1..512}.

    The TiO2 workloads take ``n_orb`` to shrink the orbital count (smaller
    profiling cases with the same positions).
    """
    if name == "cubic16":
        w = Workload(name, cubic_lattice(10.0), (16, 16, 16), 8, table_seed=0, pos_seed=0,
                     uniform_n=64)
    elif name == "tio2":
        w = Workload(name, TIO2_CELL, TIO2_GRID, kw.pop("n_orb", 768), table_seed=0,
                     pos_seed=101, uniform_n=1536)
    elif name == "tio2_batch":
        b = kw.pop("batch", 1536)
        w = Workload(name, TIO2_CELL, TIO2_GRID, kw.pop("n_orb", 768), table_seed=0,
                     pos_seed=102, n_walkers=kw.pop("n_walkers", 256), n_per_walker=1536, batch=b)
    elif name == "tio2_precision":
        w = Workload(name, TIO2_CELL, TIO2_GRID, kw.pop("n_orb", 768), table_seed=0,
                     pos_seed=103, n_walkers=kw.pop("n_walkers", 1024), n_per_walker=1536,
                     batch=1536)
    elif name == "tio2_kpoints":
        nk_axis = 4
        ks = [(i / nk_axis, j / nk_axis, k / nk_axis) for i in range(nk_axis)
              for j in range(nk_axis) for k in range(nk_axis)]
        per_k = kw.pop("per_k", 6)
        w = Workload(name, tetragonal_lattice(17.4 / 4, 11.2 / 4), (18, 18, 12), per_k * len(ks),
                     is_complex=True, table_seed=0, pos_seed=105,
                     n_walkers=kw.pop("n_walkers", 256), n_per_walker=1536,
                     batch=kw.pop("batch", 128),
                     extra={"kfrac": np.array(ks, dtype=np.float64),
                            "koffs": np.arange(0, per_k * len(ks) + 1, per_k, dtype=np.int32)},
                     pos_lattice=TIO2_CELL)
    elif name == "tio2_super_complex":
        w = Workload(name, tetragonal_lattice(34.8, 22.4), (144, 144, 96), kw.pop("n_orb", 1536),
                     is_complex=True, table_seed=0, pos_seed=104,
                     n_walkers=kw.pop("n_walkers", 512), n_per_walker=512, ragged=(1, 512),
                     extra={"spectral": True})
    else:
        raise KeyError(name)
    for k, v in kw.items():
        setattr(w, k, v)
    return w
