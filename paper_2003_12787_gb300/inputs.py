"""Seeded synthetic inputs for the elastic Space-Time Predictor.

This module holds no arithmetic of the method: it only places sample points
and draws material fields and an initial state. Both the CUDA path and the
oracle receive the arrays it returns.

Recipe (the paper's benchmark is a 3-D elastic wave problem with 9 state
quantities and 3 material parameters per node, Sec. VI; its scenario files are
not available, so seeded synthetic fields of that shape stand in for them):

* Elements: an axis-aligned grid of Gx x Gy x Gz cubes of side h, element
  index e = (ez*Gy + ey)*Gx + ex (x fastest); the first E elements in that
  order. Node (z,y,x) of element e sits at ((ex, ey, ez) + (xi_x, xi_y, xi_z))*h
  with xi the N Gauss-Legendre points on [0,1] (numpy's leggauss, used here
  only to place sample points).
* Material per node, seed ``seed_material``: rho ~ U[2,3], cp ~ U[4,6] drawn as
  two arrays of shape (E,N,N,N) in that order; cs = cp/sqrt(3).
* Initial state, seed ``seed_waves``: 4 plane waves. Direction ~ normalised
  standard normal 3-vector, radius ~ U[0,1]^(1/3) (uniform in the unit ball),
  wavevector k = 2*pi*radius*direction; amplitudes a[w,s] ~ U[0.5,1] and phases
  ph[w,s] ~ U[0,2*pi) of shape (4,9).
  q_s(x) = sum_w a[w,s] sin(k_w . x + ph[w,s]).
* Time step dt = 0.4*h / ((2N-1) * max cp).

Curvilinear elements (the paper's benchmark meshes are curvilinear and store
9 geometry parameters per node, Sec. VI): the same grid pushed through the
smooth map x_j = X_j + a/(2 pi) sin(2 pi X_{j+1}) sin(2 pi X_{j+2}) (indices
mod 3, X the Cartesian position above, a = 0.2 by default), whose Jacobian
I + a (...) is diagonally dominant for a < 1/2. Each node stores
G = (h dx/dX)^-1, the inverse Jacobian of its element's map from the
reference cube (3x3 inverse by cofactors); the state is the same plane-wave
sum evaluated at the mapped positions, and dt uses the bound 1 - 2a on the
smallest singular value of dx/dX (each row of the perturbation has two
entries of size <= a): dt = 0.4*h*(1 - 2a) / ((2N-1) * max cp).

Layouts: q [E][N][N][N][9] (z,y,x,quantity), params [E][N][N][N][3]
(rho, cp, cs), metric [E][N][N][N][3][3] (G[d][j] = dxi_d/dx_j), float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

M = 9
N_WAVES = 4


@dataclass
class Problem:
    N: int
    E: int
    h: float
    dt: float
    q: torch.Tensor       # [E][N][N][N][9] float64
    params: torch.Tensor  # [E][N][N][N][3] float64
    grid: tuple
    metric: torch.Tensor | None = None  # [E][N][N][N][3][3] float64 (curvilinear)

    @property
    def order(self) -> int:
        return self.N - 1


def sample_points(N: int, nodes: str = "gl") -> np.ndarray:
    """Positions on [0,1] where the state is sampled: Gauss-Legendre points
    (numpy's leggauss) or Gauss-Lobatto points (end points and the roots of
    P_{N-1}' from numpy's Legendre class)."""
    if nodes == "gl":
        t, _ = np.polynomial.legendre.leggauss(N)
    elif nodes == "gll":
        inner = np.polynomial.legendre.Legendre.basis(N - 1).deriv().roots().real if N > 2 else []
        t = np.concatenate([[-1.0], np.sort(inner), [1.0]])
    else:
        raise ValueError(f"unknown node family {nodes!r}")
    return (t + 1.0) / 2.0


def wave_parameters(seed_waves: int):
    rng = np.random.Generator(np.random.PCG64(seed_waves))
    d = rng.standard_normal((N_WAVES, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = rng.uniform(0.0, 1.0, N_WAVES) ** (1.0 / 3.0)
    k = 2.0 * math.pi * r[:, None] * d
    amp = rng.uniform(0.5, 1.0, (N_WAVES, M))
    phase = rng.uniform(0.0, 2.0 * math.pi, (N_WAVES, M))
    return k, amp, phase


def material(N: int, E: int, seed_material: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed_material))
    rho = rng.uniform(2.0, 3.0, (E, N, N, N))
    cp = rng.uniform(4.0, 6.0, (E, N, N, N))
    cs = cp / math.sqrt(3.0)
    return np.stack([rho, cp, cs], axis=-1)


def _grid(grid, E, h):
    """(grid, E, h) with the defaults of ``elastic_problem`` filled in."""
    if grid is None:
        if E is None:
            raise ValueError("give grid or E")
        G = max(1, math.ceil(round(E ** (1.0 / 3.0), 9)))
        while G ** 3 < E:
            G += 1
        grid = (G, G, G)
    Gx, Gy, Gz = grid
    if E is None:
        E = Gx * Gy * Gz
    if E > Gx * Gy * Gz:
        raise ValueError("E larger than the grid")
    if h is None:
        h = 1.0 / max(grid)
    return tuple(grid), E, h


def elastic_problem(N: int, grid=None, E: int | None = None, h: float | None = None,
                    seed_material: int = 1001, seed_waves: int = 1002,
                    device: str | torch.device = "cpu", nodes: str = "gl") -> Problem:
    """Build one seeded elastic STP input set.

    grid: (Gx, Gy, Gz); if omitted, a cube of side ceil(E^(1/3)).
    h: element side; default 1/max(grid). nodes: "gl" or "gll", the node
    family the state is sampled on (it must match the predictor's).
    The state is evaluated with torch on ``device`` (float64) so large inputs
    can be generated where they are used; the random draws are numpy PCG64.
    """
    grid, E, h = _grid(grid, E, h)
    Gx, Gy, Gz = grid
    params_np = material(N, E, seed_material)
    cp_max = float(params_np[..., 1].max()) if E > 0 else 5.0
    dt = 0.4 * h / ((2 * N - 1) * cp_max)
    k, amp, phase = wave_parameters(seed_waves)

    dev = torch.device(device)
    xi = torch.tensor(sample_points(N, nodes), dtype=torch.float64, device=dev)
    e = torch.arange(E, device=dev, dtype=torch.int64)
    ex = (e % Gx).to(torch.float64)
    ey = ((e // Gx) % Gy).to(torch.float64)
    ez = (e // (Gx * Gy)).to(torch.float64)
    # physical coordinates of every node, each broadcast to [E][N][N][N]
    X = ((ex[:, None] + xi[None, :]) * h)[:, None, None, :]
    Y = ((ey[:, None] + xi[None, :]) * h)[:, None, :, None]
    Z = ((ez[:, None] + xi[None, :]) * h)[:, :, None, None]
    q = torch.zeros((E, N, N, N, M), dtype=torch.float64, device=dev)
    for w in range(N_WAVES):
        kx, ky, kz = (float(v) for v in k[w])
        arg = kx * X + ky * Y + kz * Z  # [E][N][N][N] by broadcasting
        for s in range(M):
            q[..., s] += float(amp[w, s]) * torch.sin(arg + float(phase[w, s]))
    params = torch.from_numpy(params_np).to(dev)
    return Problem(N=N, E=E, h=h, dt=dt, q=q, params=params, grid=tuple(grid))


def curvilinear_problem(N: int, grid=None, E: int | None = None, h: float | None = None,
                        seed_material: int = 1001, seed_waves: int = 1002, amplitude: float = 0.2,
                        device: str | torch.device = "cpu", nodes: str = "gl") -> Problem:
    """Seeded elastic STP input set on curvilinear elements: the grid of
    ``elastic_problem`` pushed through the smooth map of the module recipe.
    Returns a Problem whose ``metric`` holds the per-node inverse Jacobians."""
    if not 0.0 <= amplitude < 0.5:
        raise ValueError("amplitude must be in [0, 0.5) for an invertible map")
    grid, E, h = _grid(grid, E, h)
    Gx, Gy, Gz = grid
    dev = torch.device(device)
    xi = torch.tensor(sample_points(N, nodes), dtype=torch.float64, device=dev)
    e = torch.arange(E, device=dev, dtype=torch.int64)
    ex = (e % Gx).to(torch.float64)
    ey = ((e // Gx) % Gy).to(torch.float64)
    ez = (e // (Gx * Gy)).to(torch.float64)
    shape = (E, N, N, N)
    X = [((ex[:, None] + xi[None, :]) * h)[:, None, None, :].expand(shape),
         ((ey[:, None] + xi[None, :]) * h)[:, None, :, None].expand(shape),
         ((ez[:, None] + xi[None, :]) * h)[:, :, None, None].expand(shape)]
    tw = 2.0 * math.pi
    sn = [torch.sin(tw * c) for c in X]
    cs_ = [torch.cos(tw * c) for c in X]
    x = [X[j] + amplitude / tw * sn[(j + 1) % 3] * sn[(j + 2) % 3] for j in range(3)]
    J = torch.zeros(shape + (3, 3), dtype=torch.float64, device=dev)  # dx_j/dX_m
    for j in range(3):
        J[..., j, j] = 1.0
        J[..., j, (j + 1) % 3] = amplitude * cs_[(j + 1) % 3] * sn[(j + 2) % 3]
        J[..., j, (j + 2) % 3] = amplitude * sn[(j + 1) % 3] * cs_[(j + 2) % 3]
    # inverse by cofactors: inv[m][j] = cof[j][m] / det
    cof = torch.empty_like(J)
    for r in range(3):
        for c in range(3):
            r1, r2, c1, c2 = (r + 1) % 3, (r + 2) % 3, (c + 1) % 3, (c + 2) % 3
            cof[..., r, c] = J[..., r1, c1] * J[..., r2, c2] - J[..., r1, c2] * J[..., r2, c1]
    det = (J[..., 0, :] * cof[..., 0, :]).sum(-1)
    metric = cof.transpose(-1, -2) / (det[..., None, None] * h)
    s_min = 1.0 - 2.0 * amplitude
    params = torch.from_numpy(material(N, E, seed_material)).to(dev)
    cp_max = float(params[..., 1].max()) if E > 0 else 5.0
    dt = 0.4 * h * s_min / ((2 * N - 1) * cp_max)
    k, amp, phase = wave_parameters(seed_waves)
    q = torch.zeros((E, N, N, N, M), dtype=torch.float64, device=dev)
    for w in range(N_WAVES):
        kx, ky, kz = (float(v) for v in k[w])
        arg = kx * x[0] + ky * x[1] + kz * x[2]
        for s in range(M):
            q[..., s] += float(amp[w, s]) * torch.sin(arg + float(phase[w, s]))
    return Problem(N=N, E=E, h=h, dt=dt, q=q, params=params, grid=grid,
                   metric=metric.contiguous())


def periodic_problem(N: int, grid, h: float | None = None, seed_material: int = 1001,
                     seed_waves: int = 1002, device: str | torch.device = "cpu",
                     nodes: str = "gl", per_node_material: bool = False) -> Problem:
    """Input set of the full ADER-DG step (predictor + corrector) on a grid that
    is periodic in every direction, box [0, Gx h] x [0, Gy h] x [0, Gz h].

    * State, seed ``seed_waves``: 4 plane waves periodic on the box. Integer
      wave numbers n ~ U{-2..2}^3 (drawn again while all three are 0),
      k = 2 pi (n_x/(Gx h), n_y/(Gy h), n_z/(Gz h)); amplitudes a[w,s] ~
      U[0.5,1] and phases ph[w,s] ~ U[0,2 pi) of shape (4,9), drawn in that
      order; q_s(x) = sum_w a[w,s] sin(k_w . x + ph[w,s]).
    * Material, seed ``seed_material``: constant inside each element (the
      paper's LOH1 benchmark is a layered medium: piecewise constant
      material), rho ~ U[2,3] and cp ~ U[4,6] per element, cs = cp/sqrt(3);
      with per_node_material, the per-node draw of ``material`` instead.
    * dt = 0.4*h / ((2N-1) * max cp), as for the predictor alone.
    """
    Gx, Gy, Gz = (int(g) for g in grid)
    E = Gx * Gy * Gz
    if h is None:
        h = 1.0 / max(Gx, Gy, Gz)
    if per_node_material:
        params_np = material(N, E, seed_material)
    else:
        rng = np.random.Generator(np.random.PCG64(seed_material))
        rho = rng.uniform(2.0, 3.0, E)
        cp = rng.uniform(4.0, 6.0, E)
        params_np = np.empty((E, N, N, N, 3))
        params_np[..., 0] = rho[:, None, None, None]
        params_np[..., 1] = cp[:, None, None, None]
        params_np[..., 2] = (cp / math.sqrt(3.0))[:, None, None, None]
    dt = 0.4 * h / ((2 * N - 1) * float(params_np[..., 1].max()))
    rng = np.random.Generator(np.random.PCG64(seed_waves))
    ks = []
    while len(ks) < N_WAVES:
        n = rng.integers(-2, 3, 3)
        if np.any(n != 0):
            ks.append(2.0 * math.pi * n / (np.array([Gx, Gy, Gz]) * h))
    amp = rng.uniform(0.5, 1.0, (N_WAVES, M))
    phase = rng.uniform(0.0, 2.0 * math.pi, (N_WAVES, M))
    dev = torch.device(device)
    xi = torch.tensor(sample_points(N, nodes), dtype=torch.float64, device=dev)
    e = torch.arange(E, device=dev, dtype=torch.int64)
    ex = (e % Gx).to(torch.float64)
    ey = ((e // Gx) % Gy).to(torch.float64)
    ez = (e // (Gx * Gy)).to(torch.float64)
    X = ((ex[:, None] + xi[None, :]) * h)[:, None, None, :]
    Y = ((ey[:, None] + xi[None, :]) * h)[:, None, :, None]
    Z = ((ez[:, None] + xi[None, :]) * h)[:, :, None, None]
    q = torch.zeros((E, N, N, N, M), dtype=torch.float64, device=dev)
    for w in range(N_WAVES):
        kx, ky, kz = (float(v) for v in ks[w])
        arg = kx * X + ky * Y + kz * Z
        for s in range(M):
            q[..., s] += float(amp[w, s]) * torch.sin(arg + float(phase[w, s]))
    params = torch.from_numpy(params_np).to(dev)
    return Problem(N=N, E=E, h=h, dt=dt, q=q, params=params, grid=(Gx, Gy, Gz))


# --- named workloads --------------------------------------------------------

def small_case() -> Problem:
    """Order 3 (N=4), 8^3 = 512 elements of side 1/8."""
    return elastic_problem(4, grid=(8, 8, 8))


def order7_case(device="cpu") -> Problem:
    """Order 7 (N=8), 32^3 = 32768 elements of side 1/32."""
    return elastic_problem(8, grid=(32, 32, 32), device=device)


def ader_order7_case(device="cpu") -> Problem:
    """Full ADER-DG step, order 7 (N=8), periodic 32^3 grid of side 1/32."""
    return periodic_problem(8, (32, 32, 32), device=device)


def order9_case(device="cpu") -> Problem:
    """Order 9 (N=10), 16384 elements on a 32x32x16 grid, side 1/32."""
    return elastic_problem(10, grid=(32, 32, 16), h=1.0 / 32, device=device)


def batched_sets_recipe(seed: int = 1003, n_sets: int = 64, n_min: int = 4, n_max: int = 12,
                        e_min: int = 64, e_max: int = 16384):
    """Sizes and seeds of the batched workload: n_sets element sets with
    N_i ~ U{n_min..n_max} and E_i = round(exp(U[ln e_min, ln e_max])) drawn from
    PCG64(seed) in that order; set i uses material/wave seeds 1001+16i,
    1002+16i on a cube grid of side ceil(E_i^(1/3)), h = 1/side, first E_i
    elements."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ns = rng.integers(n_min, n_max + 1, n_sets)
    Es = np.rint(np.exp(rng.uniform(math.log(e_min), math.log(e_max), n_sets))).astype(int)
    out = []
    for i in range(n_sets):
        E = int(Es[i])
        G = max(1, math.ceil(round(E ** (1.0 / 3.0), 9)))
        while G ** 3 < E:
            G += 1
        out.append(dict(N=int(Ns[i]), E=E, grid=(G, G, G), h=1.0 / G,
                        seed_material=1001 + 16 * i, seed_waves=1002 + 16 * i))
    return out


def batched_problems(device="cpu", **kw):
    """The batched workload's problems (see batched_sets_recipe)."""
    return [elastic_problem(r["N"], grid=r["grid"], E=r["E"], h=r["h"],
                            seed_material=r["seed_material"], seed_waves=r["seed_waves"],
                            device=device)
            for r in batched_sets_recipe(**kw)]


def served_recipe(seed: int = 1005, n_sims: int = 256, n_min: int = 4, n_max: int = 10,
                  e_min: int = 64, e_max: int = 32768):
    """Simulations of the served workload: N ~ U{n_min..n_max} and
    E = round(exp(U[ln e_min, ln e_max])) drawn from PCG64(seed) in that order;
    simulation i uses material/wave seeds 1001+16i, 1002+16i on a cube grid of
    side ceil(E^(1/3)), h = 1/side."""
    return batched_sets_recipe(seed=seed, n_sets=n_sims, n_min=n_min, n_max=n_max,
                               e_min=e_min, e_max=e_max)


def served_arrivals(n: int, rate: float = 2000.0, n_sims: int = 256, seed: int = 1006):
    """Poisson arrivals: exponential gaps of mean 1/rate seconds, then a
    simulation drawn uniformly, both from PCG64(seed) in that order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    sims = rng.integers(0, n_sims, n).astype(np.int32)
    return t, sims
