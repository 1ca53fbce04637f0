"""Full-size parity: the 256x256x512 rotor workload (33.5M cells, 5 %
turbulent inflow), the 512x512x1024 D3Q27 rotor of the storage study (FP32)
and the 1536x512x1024 wind farm (805M cells, 6 rotors), in the launch
configuration the benchmark times, compared with the FP64 oracle at sampled
cells; and a lattice at the cell-count limit.

After k steps a cell depends only on cells within a few lattice spacings
(one cell per step for collide-and-stream, at most 4 per step where the wall
model samples the velocity y_s = 2 cells off the wall), so the oracle
computes each sampled cell one by one on a sub-box of half-width 4k + 2
around it: same rotor (centre shifted to sub-box coordinates), same inflow
(each mode's phase shifted to global coordinates), same parameters, same
initial state.  Sub-boxes that reach the inlet keep the inlet as their own
open face.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

K = 4                 # steps
H = 4 * K + 2         # sub-box half-width (cells)


def _shift_modes(modes, offset):
    """Modes of a sub-box whose local coordinates are global - offset:
    a cos(k.(x+o)) + b sin(k.(x+o)) = a' cos(k.x) + b' sin(k.x)."""
    if modes is None:
        return None
    m = np.array(modes, dtype=np.float64, copy=True)
    ph = m[:, 0:3] @ np.asarray(offset, dtype=np.float64)
    c, s = np.cos(ph)[:, None], np.sin(ph)[:, None]
    a, b = m[:, 3:6].copy(), m[:, 6:9].copy()
    m[:, 3:6] = a * c + b * s
    m[:, 6:9] = b * c - a * s
    return m


def _oracle_at(wl, grids, cell):
    """(rho, u) of global cell (x, y, z) after K steps, from a sub-box oracle run."""
    a = wl.flow_axis
    lo = [cell[k] - H for k in range(3)]
    n = [2 * H + 1] * 3
    open_b = lo[a] <= 0
    if open_b:                      # keep the inlet as the sub-box's own open face
        lo[a] = 0
        n[a] = cell[a] + H + 1
    rotors = []
    for spec, grid in zip(wl.rotors, grids):
        center = tuple(spec.center[k] - lo[k] for k in range(3))
        rotors.append(O.make_rotor(grid, center=center, axis=a, omega=spec.omega(wl.u_in),
                                   phase0=spec.phase0, pitch=spec.pitch))
    off = [float(lo[k]) for k in range(3)]
    off[a] = 0.0                    # the frozen-turbulence shift acts along the flow axis
    modes = _shift_modes(wl.modes(), off)
    o = O.Oracle(n[0], n[1], n[2], q=wl.q, flow_axis=a, open_boundaries=open_b, tau_mo=wl.tau_mo,
                 c_smag=wl.c_smag, u_in=wl.u_in, eps_h=wl.eps_h, modes=modes, rotors=rotors)
    o.step(K)
    rho, u = o.fields()
    k = [cell[m] - lo[m] for m in range(3)]
    return rho[k[2], k[1], k[0]], u[:, k[2], k[1], k[0]]


def _samples(wl, grids, per_rotor_wall=10, per_rotor_solid=4, n_other=16):
    rng = np.random.default_rng(17)
    a = wl.flow_axis
    dims = wl.shape
    out = []
    for spec, grid in zip(wl.rotors, grids):
        # cells that are wall cells or force cells during the run (oracle geometry)
        rot = O.make_rotor(grid, center=spec.center, axis=a, omega=spec.omega(wl.u_in), phase0=spec.phase0)
        half = int(spec.radius) + 2
        half_a = int(np.ceil(10 * spec.radius / 64))
        rng_ax = [np.arange(int(spec.center[k]) - half, int(spec.center[k]) + half + 1) for k in range(3)]
        rng_ax[a] = np.arange(int(spec.center[a]) - half_a, int(spec.center[a]) + half_a + 1)
        cand = np.stack(np.meshgrid(*rng_ax, indexing="ij"), -1).reshape(-1, 3)
        phi, _ = O.rotor_phi(rot, K - 1, cand)
        wall = cand[(phi >= 0) & (phi < 1)]
        solid = cand[phi < 0]
        out += [tuple(int(c) for c in v) for v in wall[rng.choice(len(wall), per_rotor_wall, replace=False)]]
        out += [tuple(int(c) for c in v) for v in solid[rng.choice(len(solid), per_rotor_solid, replace=False)]]
    # inlet-adjacent planes and random cells
    for k in range(n_other):
        c = [int(rng.integers(H, dims[m] - H)) for m in range(3)]
        if k < n_other // 2:
            c[a] = 1 + k % 3
        out.append(tuple(c))
    return out


def _run_and_compare(wl):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu-marked tests")
    from paper_2510_13726_b300.build import build
    build()
    from paper_2510_13726_b300 import Lattice
    grids = wl.blade_grids()
    lat = Lattice.from_workload(wl)          # the benchmark's launch configuration
    lat.step(K)
    samples = _samples(wl, grids)
    idx = torch.tensor([[c[2], c[1], c[0]] for c in samples], device=lat.device)
    rho_t, u_t = lat.fields()
    rho = rho_t[idx[:, 0], idx[:, 1], idx[:, 2]].cpu().numpy()
    u = u_t[:, idx[:, 0], idx[:, 1], idx[:, 2]].cpu().numpy()
    del rho_t, u_t
    lat.close()
    torch.cuda.empty_cache()
    worst_u = worst_r = 0.0
    for j, cell in enumerate(samples):
        ro, uo = _oracle_at(wl, grids, cell)
        eu = float(np.abs(u[:, j] - uo).max()) / wl.u_in
        er = abs(float(rho[j]) - ro)
        worst_u, worst_r = max(worst_u, eu), max(worst_r, er)
        assert eu <= 1e-5 and er <= 1e-6, (cell, u[:, j], uo, rho[j], ro)
    print(f"{wl.name} sampled parity ({len(samples)} cells): max |du|/U = {worst_u:.2e}, "
          f"max |drho| = {worst_r:.2e}")


def test_fullsize_rotor256_sampled_parity():
    _run_and_compare(W.workload("rotor256"))


def test_fullsize_rotor1024_q27_sampled_parity():
    """The storage-study size in FP32 (512x512x1024 D3Q27, 268M cells, R = 128,
    TSR 7): sampled cells at the rotor and near the inlet."""
    _run_and_compare(W.workload("rotor1024_q27"))


def test_fullsize_farm_sampled_parity():
    """Wind-farm scale on one GPU (1536x512x1024, 805M cells, 3x2 rotors, flow
    along x): sampled cells at every rotor and near the inlet."""
    _run_and_compare(W.workload("farm"))


def test_maximum_size_lattice():
    """Near the 2^31 - 1 cell limit: 1023 x 1024 x 2049 = 2,146,434,048 cells,
    BF16 storage (81.6 GB).  A Taylor-Green field in (x, y), uniform in z,
    evolves identically in every z slice; nx odd keeps one cell per thread, so
    every cell runs the same arithmetic and the slices at the end of the index
    range equal a 4-slice lattice bit for bit after steps of both parities."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu-marked tests")
    from paper_2510_13726_b300.build import build
    build()
    import paper_2510_13726_b300 as P
    nx, ny, nz = 1023, 1024, 2049
    assert nx * ny * nz < 2 ** 31 - 1
    kw = dict(storage="bf16s", open_boundaries=False, tau_mo=0.8, c_smag=0.1, u_in=0.0, wall_model=False,
              mass_check_every=0)

    def tgv(n_z, dev):
        x = torch.arange(nx, device=dev, dtype=torch.float32) * (2 * np.pi / nx)
        y = torch.arange(ny, device=dev, dtype=torch.float32) * (2 * np.pi / ny)
        ux = 0.03 * torch.sin(x)[None, :] * torch.cos(y)[:, None]
        uy = -0.03 * torch.cos(x)[None, :] * torch.sin(y)[:, None]
        u = torch.stack([ux, uy, torch.zeros_like(ux)])[:, None].expand(3, n_z, ny, nx)
        return u.contiguous()

    small = P.Lattice(nx, ny, 4, **kw)
    small.init_fields(u=tgv(4, small.device))
    small.step(5)
    ref = small.fields()[1][:, 0].clone()
    del small
    big = P.Lattice(nx, ny, nz, **kw)
    big.init_fields(u=tgv(nz, big.device))
    m0 = big.mass()
    big.step(5)
    _, u = big.fields()
    for z in (nz - 1, nz - 2, nz // 2, 0):
        assert torch.equal(u[:, z], ref), z
    del u
    assert abs(big.mass() - m0) <= 1e-6 * m0
    big.close()
    torch.cuda.empty_cache()
