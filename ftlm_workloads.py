"""Seeded synthetic spin systems (inputs only).

This module holds the geometry and the random coupling draws of the
benchmark systems and nothing of the method's arithmetic: no Hamiltonian
terms, no basis, no Lanczos.  Both the CUDA library's tests/benchmark and
the oracle's tests build their inputs from here, so the two sides see the
same numbers without sharing any code of the method.

Each system is a dict with keys ``two_s`` [n] (int, 2s), ``J`` [n][n] (K,
upper triangle used, H uses 2J), ``d_ion`` [n] (K) or None, ``e_axes`` [n][3]
or None, ``g``, ``B`` [3] (Tesla), ``pos`` [n][3] (Angstrom) or None, and a
``name``.

Geometry readings (the workload list gives lattice names only):
* ring: site i at angle 2 pi i / N, radius r, z = 0; a tilted axis leans
  30 degrees from z toward the outward radial direction;
* L_x x L_y lattice: site i = x + L_x * y, spacing a, z = 0, nearest
  neighbours along x and y (open boundaries);
* 2 x 13 ladder: legs of 13 sites along x, rungs along y, i = x + 13 * y;
* chain: sites along x with spacing a;
* random couplings: numpy ``default_rng(seed).uniform`` over the bonds in
  lexicographic (i < j) order; random axes: isotropic on the sphere from
  ``default_rng(seed).normal`` normalised;
* field directions on a Fibonacci sphere: z_k = 1 - (2k+1)/K,
  phi_k = k pi (3 - sqrt 5);
* Mn9-like centred cube (Sec. III.C; the published couplings are not
  available here, so the values below are synthetic): a spin-5/2 at the
  centre, eight spin-2 at the vertices of a cube of edge a (top square
  z = +a/2, bottom z = -a/2, vertex k at azimuth 45 + 90 k degrees); J_c
  centre-vertex, J_s nearest neighbours within the top and within the
  bottom square, J_e the vertical edges; each vertex has an easy axis
  (d < 0) tilted 30 degrees from z, at azimuth +10 degrees (top) or -10
  degrees (bottom) from the x axis; powder average over the 10 directions
  through the vertices of a dodecahedron, one of each antipodal pair
  (B and -B give the same thermodynamics).
"""
from __future__ import annotations

import numpy as np

DEFAULT_T = 0.05 * 1000.0 ** (np.arange(40) / 39.0)   # 40 log-spaced points 0.05 .. 50 K


def temperatures(nT: int = 40, Tmin: float = 0.05, Tmax: float = 50.0) -> np.ndarray:
    return Tmin * (Tmax / Tmin) ** (np.arange(nT) / (nT - 1))


def _system(name, two_s, J, pos, B, g=2.0, d_ion=None, e_axes=None):
    n = len(two_s)
    return {
        "name": name,
        "two_s": np.asarray(two_s, dtype=np.int32),
        "J": np.asarray(J, dtype=np.float64).reshape(n, n),
        "d_ion": None if d_ion is None else np.asarray(d_ion, dtype=np.float64),
        "e_axes": None if e_axes is None else np.asarray(e_axes, dtype=np.float64).reshape(n, 3),
        "g": float(g),
        "B": np.asarray(B, dtype=np.float64).reshape(3),
        "pos": None if pos is None else np.asarray(pos, dtype=np.float64).reshape(n, 3),
    }


def lattice_positions(Lx: int, Ly: int, a: float) -> np.ndarray:
    pos = np.zeros((Lx * Ly, 3))
    for y in range(Ly):
        for x in range(Lx):
            pos[x + Lx * y] = (a * x, a * y, 0.0)
    return pos


def lattice_bonds(Lx: int, Ly: int):
    """Nearest-neighbour bonds (i, j), i < j, of an open Lx x Ly lattice, sorted."""
    bonds = []
    for y in range(Ly):
        for x in range(Lx):
            i = x + Lx * y
            if x + 1 < Lx:
                bonds.append((i, i + 1))
            if y + 1 < Ly:
                bonds.append((i, i + Lx))
    return sorted(bonds)


def ring(N=6, two_s=2, radius=3.0, J=1.0, d=-5.0, tilt_deg=30.0, B=1.0, Bdir=(1, 1, 1), dipolar=True, g=2.0):
    """Ring in the xy-plane, nearest-neighbour J, tilted single-ion axes."""
    ang = 2 * np.pi * np.arange(N) / N
    pos = np.stack([radius * np.cos(ang), radius * np.sin(ang), np.zeros(N)], axis=1)
    t = np.deg2rad(tilt_deg)
    axes = np.stack([np.sin(t) * np.cos(ang), np.sin(t) * np.sin(ang), np.cos(t) * np.ones(N)], axis=1)
    Jm = np.zeros((N, N))
    for i in range(N):
        j = (i + 1) % N
        a, b = min(i, j), max(i, j)
        Jm[a, b] = J
    bd = np.asarray(Bdir, dtype=np.float64)
    bd = bd / np.linalg.norm(bd)
    return _system(f"ring N={N} 2s={two_s}", [two_s] * N, Jm, pos if dipolar else None, B * bd, g=g,
                   d_ion=np.full(N, d), e_axes=axes)


def square_lattice(Lx, Ly, a=3.5, Jlow=0.5, Jhigh=1.5, seed=1, B=0.5, Bdir=(0, 0.6, 0.8), two_s=1, dipolar=True,
                   g=2.0):
    """Open Lx x Ly lattice, nearest-neighbour J_ij ~ U[Jlow, Jhigh] (seeded)."""
    n = Lx * Ly
    rng = np.random.default_rng(seed)
    Jm = np.zeros((n, n))
    for (i, j) in lattice_bonds(Lx, Ly):
        Jm[i, j] = rng.uniform(Jlow, Jhigh)
    bd = np.asarray(Bdir, dtype=np.float64)
    bd = bd / np.linalg.norm(bd)
    return _system(f"{Lx}x{Ly} lattice 2s={two_s}", [two_s] * n, Jm,
                   lattice_positions(Lx, Ly, a) if dipolar else None, B * bd, g=g)


def ladder(legs=13, a=3.5, J_rung=1.0, J_leg=0.6, B=0.2, Bdir=(0, 0, 1), dipolar=True, g=2.0):
    """Open 2 x legs ladder: legs along x, rungs along y, i = x + legs * y."""
    n = 2 * legs
    pos = lattice_positions(legs, 2, a)
    Jm = np.zeros((n, n))
    for (i, j) in lattice_bonds(legs, 2):
        Jm[i, j] = J_rung if j - i == legs else J_leg
    bd = np.asarray(Bdir, dtype=np.float64)
    bd = bd / np.linalg.norm(bd)
    return _system(f"2x{legs} ladder", [1] * n, Jm, pos if dipolar else None, B * bd, g=g)


def random_axes(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def fibonacci_directions(K=8):
    k = np.arange(K)
    z = 1.0 - (2 * k + 1) / K
    phi = k * np.pi * (3.0 - np.sqrt(5.0))
    rho = np.sqrt(1.0 - z * z)
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def chain(N, two_s=2, a=4.0, J=0.8, d=-3.0, axes_seed=3, B=1.0, Bdir=(0, 0, 1), dipolar=True, g=2.0, max_sites=12):
    """Open chain along x, uniform J, single-ion axes isotropic on the sphere
    (the first N of ``max_sites`` seeded draws, so chains of different length
    share their first axes)."""
    pos = np.stack([a * np.arange(N), np.zeros(N), np.zeros(N)], axis=1)
    Jm = np.zeros((N, N))
    for i in range(N - 1):
        Jm[i, i + 1] = J
    axes = random_axes(max(max_sites, N), axes_seed)[:N]
    bd = np.asarray(Bdir, dtype=np.float64)
    bd = bd / np.linalg.norm(bd)
    return _system(f"chain N={N} 2s={two_s}", [two_s] * N, Jm, pos if dipolar else None, B * bd, g=g,
                   d_ion=np.full(N, d), e_axes=axes)


# --- the benchmark systems -------------------------------------------------

def ring6_s1():
    """N=6 s=1 ring, r=3 A, J=1 K, d=-5 K tilted 30 deg, B=1 T || (1,1,1), dipolar (d=729)."""
    return ring()


def lattice4x4():
    """Open 4x4 s=1/2, a=3.5 A, J ~ U[0.5,1.5] K (seed 1), B=0.5 T || (0,.6,.8), dipolar (d=65,536)."""
    return square_lattice(4, 4, Jlow=0.5, Jhigh=1.5, seed=1, B=0.5, Bdir=(0, 0.6, 0.8))


def lattice4x5():
    """Open 4x5 s=1/2, a=3.5 A, J ~ U[-1,1.5] K (seed 2), B=2 T || (1,0,1), dipolar (d=1,048,576)."""
    return square_lattice(4, 5, Jlow=-1.0, Jhigh=1.5, seed=2, B=2.0, Bdir=(1, 0, 1))


def ladder2x13():
    """Open 2x13 s=1/2 ladder, rung 1.0 K, leg 0.6 K, B=0.2 T || z, dipolar (d=67,108,864)."""
    return ladder()


def chain_batch():
    """24 instances: s=1 chains N in {10,11,12} x 8 Fibonacci field directions at 1 T."""
    out = []
    for N in (10, 11, 12):
        for bd in fibonacci_directions(8):
            out.append(chain(N, Bdir=bd))
    return out


def dodecahedron_directions():
    """10 unit vectors: one vertex of each antipodal pair of a regular
    dodecahedron, (1,1,1)-type and the cyclic (0, 1/phi, phi) family."""
    ph = (1 + np.sqrt(5.0)) / 2
    v = [(1, 1, 1), (1, 1, -1), (1, -1, 1), (1, -1, -1),
         (0, 1 / ph, ph), (0, 1 / ph, -ph), (1 / ph, ph, 0), (1 / ph, -ph, 0), (ph, 0, 1 / ph), (ph, 0, -1 / ph)]
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def mn9(Bdir=(0, 0, 1), B=1.0, vertices=8, a=3.6, Jc=-1.2, Js=0.4, Je=0.25, D=-1.5):
    """Mn9-like centred cube: site 0 spin 5/2 at the centre, sites 1..8 spin 2
    at the cube vertices (1-4 top, 5-8 bottom); `vertices` < 8 keeps the first
    ones (a smaller test system).  d = 6 * 5^vertices (2,343,750 for 8)."""
    n = 1 + vertices
    pos = np.zeros((n, 3))
    axes = np.zeros((n, 3))
    d_ion = np.zeros(n)
    for k in range(vertices):
        top = k < 4
        az = np.deg2rad(45 + 90 * (k % 4))
        pos[1 + k] = (a / np.sqrt(2) * np.cos(az), a / np.sqrt(2) * np.sin(az), a / 2 if top else -a / 2)
        phi = np.deg2rad(10 if top else -10)
        th = np.deg2rad(30)
        axes[1 + k] = (np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th))
        d_ion[1 + k] = D
    axes[0] = (0, 0, 1)
    J = np.zeros((n, n))
    for k in range(vertices):
        J[0, 1 + k] = Jc
    for k in range(vertices):
        for l in range(k + 1, vertices):
            same = (k < 4) == (l < 4)
            if same and (l - k) % 4 in (1, 3):     # neighbours within a square
                J[1 + k, 1 + l] = Js
            elif not same and l - k == 4:          # vertical edge
                J[1 + k, 1 + l] = Je
    bd = np.asarray(Bdir, dtype=np.float64)
    bd = bd / np.linalg.norm(bd)
    return _system(f"mn9_{vertices}", [5] + [4] * vertices, J, pos, B * bd, g=2.0, d_ion=d_ion, e_axes=axes)


def mn9_powder():
    """The Mn9-like system at 1 T along each of the 10 dodecahedron directions."""
    return [mn9(Bdir=u) for u in dodecahedron_directions()]


WORKLOADS = {
    "ring6_s1": dict(system=ring6_s1, R=10, M=80, dtype="c128", seed=0),
    "lattice4x4": dict(system=lattice4x4, R=50, M=150, dtype="c128", seed=1),
    "lattice4x5": dict(system=lattice4x5, R=64, M=200, dtype="c64", seed=2),
    "chains_s1_x24": dict(system=chain_batch, R=16, M=120, dtype="c64", seed=3),
    "ladder2x13": dict(system=ladder2x13, R=4, M=300, dtype="c64", seed=4),
    "mn9_powder": dict(system=mn9_powder, R=8, M=40, dtype="c64", seed=5),
}
