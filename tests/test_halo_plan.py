"""The split box's halo exchange as data (grf_halo_plan), on the CPU:
  * applied to patches cut from a box, the plan fills every ghost point with the box's value
    there, bit for bit: the periodic wrap of a periodic box (decompositions with patches
    narrower than the 3 ghost layers, single-patch axes that wrap onto themselves), and in a
    frozen box the ghosts inside the box while those outside it stay untouched;
  * every ghost point is written by exactly one block;
  * across two gloo ranks, each holding half of the patches, the point-to-point exchange by the
    plan gives the same patches as the single-process application.
"""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

import grf_inputs as gi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def grf():
    from paper_2309_06225_gb300 import build
    build.build()
    import paper_2309_06225_gb300 as g
    try:
        g.lib()
    except OSError as e:  # libcudart missing on a machine without the toolkit
        pytest.skip(f"cannot load libgrf.so here: {e}")
    return g


CASES = [((12, 12, 12), (2, 2, 2), gi.BC_PERIODIC), ((10, 7, 9), (3, 1, 2), gi.BC_PERIODIC),
         ((8, 8, 8), (4, 4, 4), gi.BC_PERIODIC), ((5, 4, 3), (1, 1, 1), gi.BC_PERIODIC),
         ((9, 8, 7), (2, 3, 1), gi.BC_FROZEN), ((6, 5, 7), (3, 5, 2), gi.BC_FROZEN)]


def setup_case(grf, orc, n, p, bc, seed=0):
    """The box (ghosts valid: wrapped, or frozen random values), the level, the patch geometries
    and offsets, and patches holding the box's interior with NaN ghosts."""
    box = gi.Box(*n, 0.3, -1.0, -1.0, -1.0, bc=bc)
    rng = np.random.default_rng(seed)
    s = rng.normal(size=box.shape)
    if bc == gi.BC_PERIODIC:
        orc.fill_ghosts(box, s)
    level = grf.patch_level(grf.box_like(box), *p)
    patches, offs = [], []
    for q in range(p[0] * p[1] * p[2]):
        pb = grf.grf_patch_box(level, q)
        off = [int(round((c - c0) / box.dx)) for c, c0 in ((pb.x0, box.x0), (pb.y0, box.y0), (pb.z0, box.z0))]
        a = np.full((27, pb.nz + 6, pb.ny + 6, pb.pitch), np.nan)
        a[:, 3:3 + pb.nz, 3:3 + pb.ny, 3:3 + pb.nx] = s[:, 3 + off[2]:3 + off[2] + pb.nz,
                                                        3 + off[1]:3 + off[1] + pb.ny,
                                                        3 + off[0]:3 + off[0] + pb.nx]
        patches.append(a)
        offs.append((off, (pb.nx, pb.ny, pb.nz)))
    return box, s, level, patches, offs


def expected_patch(box, s, off, ext, pitch):
    """The box's values over the patch's ghosted block; a frozen box's ghosts outside the box are
    not written by an exchange (NaN here, as the patches start)."""
    (ox, oy, oz), (nx, ny, nz) = off, ext
    e = np.full((27, nz + 6, ny + 6, pitch), np.nan)
    e[:, :, :, :nx + 6] = s[:, oz:oz + nz + 6, oy:oy + ny + 6, ox:ox + nx + 6]
    if box.bc == gi.BC_FROZEN:
        k, j, i = np.meshgrid(np.arange(nz + 6) + oz - 3, np.arange(ny + 6) + oy - 3, np.arange(nx + 6) + ox - 3,
                              indexing="ij")
        outside = (i < 0) | (i >= box.nx) | (j < 0) | (j >= box.ny) | (k < 0) | (k >= box.nz)
        e[:, :, :, :nx + 6][:, outside] = np.nan
    return e


@pytest.mark.parametrize("n,p,bc", CASES)
def test_plan_fills_every_ghost_with_the_box_value(grf, orc, n, p, bc):
    from paper_2309_06225_gb300 import halo
    box, s, level, patches, offs = setup_case(grf, orc, n, p, bc)
    plan = grf.grf_halo_plan(level)
    halo.apply_plan(plan, patches)
    for q, (off, ext) in enumerate(offs):
        assert np.array_equal(patches[q], expected_patch(box, s, off, ext, patches[q].shape[3]), equal_nan=True), q


@pytest.mark.parametrize("n,p,bc", CASES)
def test_plan_writes_each_ghost_point_once(grf, orc, n, p, bc):
    box, s, level, patches, offs = setup_case(grf, orc, n, p, bc)
    hits = [np.zeros(a.shape[1:], dtype=int) for a in patches]
    for b in grf.grf_halo_plan(level):
        hits[b.dst][b.dst_k:b.dst_k + b.nk, b.dst_j:b.dst_j + b.nj, b.dst_i:b.dst_i + b.ni] += 1
        (sx, sy, sz), (nx, ny, nz) = offs[b.src][0], offs[b.src][1]
        # sources lie inside the source patch's interior
        assert 3 <= b.src_i and b.src_i + b.ni <= 3 + nx
        assert 3 <= b.src_j and b.src_j + b.nj <= 3 + ny
        assert 3 <= b.src_k and b.src_k + b.nk <= 3 + nz
    for q, (off, ext) in enumerate(offs):
        want = np.isnan(patches[q][0]).astype(int)  # ghost points (NaN before the exchange) ...
        e = expected_patch(box, s, off, ext, patches[q].shape[3])[0]
        want[np.isnan(e)] = 0                       # ... except those no exchange writes
        assert np.array_equal(hits[q], want), q


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, case, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as dist
    import oracle
    import paper_2309_06225_gb300 as grf
    from paper_2309_06225_gb300 import halo
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, p, bc = case
    box, s, level, patches, offs = setup_case(grf, oracle, n, p, bc)
    plan = grf.grf_halo_plan(level)
    owner = [qq % world for qq in range(len(patches))]
    local = {qq: torch.from_numpy(patches[qq]) for qq in range(len(patches)) if owner[qq] == rank}
    halo.exchange(plan, local, owner, rank)
    ok = all(np.array_equal(local[qq].numpy(), expected_patch(box, s, offs[qq][0], offs[qq][1], patches[qq].shape[3]),
                            equal_nan=True) for qq in local)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ok, len(local)))


@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[4]])
def test_two_gloo_ranks_exchange_by_the_plan(case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, case, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=180)
    assert all(pr.exitcode == 0 for pr in procs), [pr.exitcode for pr in procs]
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert all(ok for _, ok, _ in got), got
    assert sum(nl for _, _, nl in got) == case[1][0] * case[1][1] * case[1][2]
