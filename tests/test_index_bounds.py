"""Bounds of the step kernels' shared-memory and global indexing, checked on
the CPU over a dense set of grids (a model of the kernels' index arithmetic,
like tests/test_transfer_scan.py's model of the transfer scan).

The register-path kernel (csrc/sfd_step_reg.cuh) carves each warp's (or warp
group's) shared-memory region into arrays that start two words into a slot:
2 transverse slots of 32 MU + 4 words (MU rows per lane) and 12 longitudinal
slots of 32 m_z + 4 words (18 when the longitudinal matrix is factored
instead of folded into the sweeps), so array a accepts indices -2 .. slot-3.
Every index the kernel forms is a function of the lane, the row within the
lane and the grid (N_t, N_l); this test enumerates those functions for every
lane and row and asserts that each lands inside its array, that the carved
total equals the host's region size (warp_smem_floats, which launches and
string creation check against the device's shared memory), and that global
reads and writes stay inside the host-allocated state, output and
trajectory arrays.  The host-side rules (rows per lane, region size) are
restated from sfd_api.cu (rows_per_lane) and sfd_types.h (warp_smem_floats);
a change to the kernels' carving or index arithmetic must be mirrored here,
as for the transfer-scan model."""

import numpy as np
import pytest

WARP = 32


def rows_per_lane(n):
    """Odd m with 32 m >= n + 1 (host rule of sfd_api.cu)."""
    m = max(1, (n + 1 + WARP - 1) // WARP)
    return m if m % 2 else m + 1


def region_floats(m_u, m_z, z_jacobi):
    """warp_smem_floats of sfd_types.h for the register path."""
    ru = WARP * m_u + 4
    rz = WARP * m_z + 4 if m_z > 0 else 0
    return 2 * ru + (12 if z_jacobi else 18) * rz


def transfer_maps(n_t, n_l, m_u):
    """TMIs / TMWs of every transverse row (pad rows: node N_l + 1, weight 0)."""
    n_u = n_t - 1
    rows = np.arange(WARP * m_u)
    pos = (rows + 1) * n_l
    mm = np.where(rows < n_u, pos // n_t, n_l + 1)
    return rows, mm


def check_grid(n_t, n_l, z_jacobi, group=1):
    n_u, n_z = n_t - 1, (n_l - 1 if n_l > 1 else 0)
    m_u, m_z = rows_per_lane(n_u), (rows_per_lane(n_z) if n_z > 0 else 0)
    if m_u > 9:
        return False        # the shared-memory path (its own test below)
    RU, RZ = WARP * m_u + 4, (WARP * m_z + 4 if m_z else 0)
    u_lo, u_hi = -2, RU - 3          # valid indices of a transverse array
    z_lo, z_hi = -2, RZ - 3          # ... of a longitudinal array
    # carving: 2 transverse + 12 or 18 longitudinal slots, zeroed [0, total)
    total = 2 * RU + ((12 if z_jacobi else 18) * RZ if m_z else 0)
    assert total == region_floats(m_u, m_z, z_jacobi)
    # transverse rows of a lane: i = lane MU + r, r < MU
    rows = np.arange(WARP * m_u)
    assert rows.min() >= u_lo and rows.max() <= u_hi
    assert rows.max() >= n_u       # the last real row has a zero pad row to its right
    if m_z == 0:
        return True
    # TMIs / TMWs at the transverse rows; the interpolation reads A[mm - 1], A[mm]
    rows, mm = transfer_maps(n_t, n_l, m_u)
    assert mm.min() - 1 >= z_lo and mm.max() <= z_hi
    real = rows < n_u
    assert mm[real].max() <= n_l - 1 and mm[real].min() >= 0
    # the scan stores S0[m], S1[m + 1] from real rows only; spreadS reads [i + 1]
    assert mm[real].max() + 1 <= z_hi
    # longitudinal rows visited by z_rows: lane + 32 k, k < m_z, split by the group
    for pw in range(group):
        zi = np.array([lane + WARP * k for lane in range(WARP) for k in range(pw, m_z, group)], int)
        if zi.size == 0:
            continue
        assert zi.min() - 1 >= z_lo and zi.max() + 1 <= z_hi            # Z[i -+ 1], AZ[i -+ 1]
        assert zi.max() + 1 <= z_hi                                       # S0[i + 1], S1[i + 1]
    # factored longitudinal solve: rows lane m_z + r
    zf = np.array([lane * m_z + r for lane in range(WARP) for r in range(m_z)], int)
    assert zf.min() >= z_lo and zf.max() <= z_hi
    # the state loads and stores touch global z[i] for i < n_z only
    assert n_z <= WARP * m_z - 1
    return True


def grids():
    """Every N_t 2..288 (register path) against N_l spanning the ratios the
    grid rule produces (N_l from 1 to 16 N_t) plus the largest grids."""
    out = []
    for n_t in range(2, 289, 3):
        for n_l in sorted({1, 2, 3, max(1, n_t // 7), max(1, n_t // 3), n_t - 1, n_t, n_t + 1, 2 * n_t,
                           4 * n_t + 3, 16 * n_t}):
            out.append((n_t, n_l))
    return out


def test_register_path_indexing_in_bounds():
    checked = 0
    for n_t, n_l in grids():
        for zj in (True, False):
            for group in (1, 2, 4):
                checked += check_grid(n_t, n_l, zj, group)
    assert checked > 5000


def test_group_exchange_cells_in_bounds():
    """Warp groups exchange each lane's four convergence maxima through
    xcell[buffer * 512 + warp * 128 + {0, 32, 64, 96} + lane] of a 1024-float
    cell per group (two alternating buffers)."""
    idx = [b * 512 + pw * 128 + off + lane for b in (0, 1) for pw in range(4) for off in (0, 32, 64, 96)
           for lane in range(WARP)]
    assert min(idx) >= 0 and max(idx) <= 1023 and len(set(idx)) == len(idx)


@pytest.mark.parametrize("n_samples", [1, 31, 32, 33, 96000])
def test_output_and_trajectory_writes_in_bounds(n_samples):
    """Output: every 32 samples lanes write out[opos - 32 + lane], the tail
    out[opos - rem + lane] for lane < rem: exactly the indices 0 .. n - 1,
    each once.  Trajectory record of step k: [u | D | z | Dz | 2 scalars] at
    k * stride, stride = 4-aligned 2 n_u + 2 n_z + 2 (sfd_tape.cuh)."""
    written = []
    opos = 0
    for _ in range(n_samples):
        opos += 1
        if opos % WARP == 0:
            written += [opos - WARP + lane for lane in range(WARP)]
    rem = opos % WARP
    written += [opos - rem + lane for lane in range(rem)]
    assert sorted(written) == list(range(n_samples))
    for n_u, n_z in [(1, 0), (31, 5), (100, 799), (287, 0)]:
        stride = -(-(2 * n_u + 2 * n_z + 2) // 4) * 4
        assert 2 * n_u + 2 * n_z + 1 < stride


def smem_region_floats(m_u, m_z):
    """warp_smem_floats for the shared-memory path (19 transverse and 15
    longitudinal arrays)."""
    ru = WARP * m_u + 4
    rz = WARP * m_z + 4 if m_z > 0 else 0
    return 19 * ru + 15 * rz


def test_shared_memory_path_indexing_in_bounds():
    """The shared-memory path keeps every per-row array in the region: rows
    lane m + r, neighbours to distance 2 (the fourth difference) on the
    transverse side and 1 on the longitudinal side, the transfer maps as
    above; arrays also start two words into slots of 32 m + 4 words."""
    checked = 0
    for n_t in range(289, 4001, 37):
        for n_l in (1, 2, n_t // 5, n_t, 3 * n_t):
            n_u, n_z = n_t - 1, (n_l - 1 if n_l > 1 else 0)
            m_u, m_z = rows_per_lane(n_u), (rows_per_lane(n_z) if n_z > 0 else 0)
            RU = WARP * m_u + 4
            rows = np.array([lane * m_u + r for lane in range(WARP) for r in range(m_u)])
            assert rows.min() - 2 >= -2 and rows.max() + 2 <= RU - 3   # U[i -+ 2] inside the array
            assert rows.max() >= n_u
            if m_z:
                RZ = WARP * m_z + 4
                _, mm = transfer_maps(n_t, n_l, m_u)
                assert mm.min() - 1 >= -2 and mm.max() <= RZ - 3
                zr = np.array([lane * m_z + r for lane in range(WARP) for r in range(m_z)])
                assert zr.min() - 1 >= -2 and zr.max() + 1 <= RZ - 3
            assert smem_region_floats(m_u, m_z) >= 19 * RU
            checked += 1
    assert checked > 400


def test_host_rules_match_the_library():
    """Every grid the library's host rule (sfd_grid) gives random strings
    has, under the rows-per-lane rule restated here, a zero pad row to the
    right of its last real row."""
    from paper_2311_18505_gb300 import sfd
    from paper_2311_18505_gb300 import workloads as W
    rng = np.random.default_rng(5)
    for _ in range(200):
        d = W.random_string(rng, f0_lo=20.0, f0_hi=2000.0, seconds=0.01)
        n_t, n_l = sfd.sfd_grid(sfd.params_from_dict(d))
        n_u = n_t - 1
        assert rows_per_lane(n_u) * WARP >= n_u + 1
