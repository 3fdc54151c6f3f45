"""Partitions (Sec. 4.2), host side: the space-filling-curve partitioner, the
owned + halo local meshes, and that the parts' block rows together are
exactly the whole mesh's pattern, once each.  Also run as two gloo ranks,
each building only its own part."""
import os
import socket

import numpy as np
import pytest

from paper_2007_04881_gb300 import configs, dg

from .helpers import dg_problem


def _blocks_full(wl):
    info, row_ptr, col, blk_off = dg.dg_mesh_check(wl.mesh, wl.p, wl.a, dg_problem(wl), pattern=True)
    out = {}
    for r in range(info.ne):
        for bk in range(row_ptr[r], row_ptr[r + 1]):
            out[(r, int(col[bk]))] = int(blk_off[bk + 1] - blk_off[bk])
    return out


def _blocks_part(wl, part, k):
    pc = dg.dg_part_check(wl.mesh, wl.p, wl.a, dg_problem(wl), part, k)
    eg, own, rp, col, bo = pc["elem_global"], pc["owned"], pc["row_ptr"], pc["col"], pc["blk_off"]
    assert np.all(np.diff(eg) > 0)  # local order = global order
    assert pc["nowned"] == int(np.sum(part == k)) == int(own.sum())
    assert set(eg[own == 1].tolist()) == set(np.flatnonzero(part == k).tolist())
    out = {}
    for r in range(pc["info"].ne):
        if not own[r]:
            assert rp[r + 1] == rp[r]  # halo rows are empty
            continue
        for bk in range(rp[r], rp[r + 1]):
            out[(int(eg[r]), int(eg[col[bk]]))] = int(bo[bk + 1] - bo[bk])
    # the load vector has entries for owned elements only
    assert pc["info"].ndofs == sum(int(dg_nb(wl.mesh.dim, wl.p[e])) for e in np.flatnonzero(part == k))
    return out


def dg_nb(dim, p):
    p = int(p)
    return (p + 1) * (p + 2) // 2 if dim == 2 else (p + 1) * (p + 2) * (p + 3) // 6


@pytest.fixture(scope="module")
def wl2():
    return configs.small2d(400, 71, 1, 4, b=(1.0, 0.5), c=1.0)


@pytest.fixture(scope="module")
def wl3():
    return configs.small3d(6, 60, 72, 1, 3)


@pytest.mark.parametrize("nparts", [1, 2, 3, 7])
def test_partition_covers_and_balances(wl2, nparts):
    pb = dg_problem(wl2)
    part = dg.dg_partition(wl2.mesh, wl2.p, wl2.a, pb, nparts)
    assert part.min() == 0 and part.max() == nparts - 1
    assert np.array_equal(part, dg.dg_partition(wl2.mesh, wl2.p, wl2.a, pb, nparts))  # deterministic
    # cost per part within one element's cost of the mean
    m = wl2.mesh
    nsub = np.diff(m.elem_vptr)
    n = (wl2.p.astype(np.int64) + 1) * (wl2.p + 2) // 2
    w = nsub * (wl2.p.astype(np.int64) + 2) ** 2 * n * n
    cost = np.bincount(part, weights=w, minlength=nparts)
    assert np.all(np.abs(cost - w.sum() / nparts) <= w.max())


def test_partition_rejects_bad_counts(wl2):
    pb = dg_problem(wl2)
    for bad in (0, -1, wl2.mesh.ne + 1):
        with pytest.raises(dg.DGError):
            dg.dg_partition(wl2.mesh, wl2.p, wl2.a, pb, bad)
    part = np.zeros(wl2.mesh.ne, np.int32)
    with pytest.raises(dg.DGError):
        dg.dg_part_check(wl2.mesh, wl2.p, wl2.a, pb, part, 1)  # part 1 owns nothing


@pytest.mark.parametrize("which,nparts", [("2d", 3), ("2d", 5), ("3d", 4)])
def test_parts_union_is_whole_pattern(wl2, wl3, which, nparts):
    wl = wl2 if which == "2d" else wl3
    full = _blocks_full(wl)
    part = dg.dg_partition(wl.mesh, wl.p, wl.a, dg_problem(wl), nparts)
    seen = {}
    for k in range(nparts):
        for key, size in _blocks_part(wl, part, k).items():
            assert key not in seen  # every block has one owner
            seen[key] = size
    assert seen == full


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        wl = configs.small2d(400, 71, 1, 4, b=(1.0, 0.5), c=1.0)
        part = dg.dg_partition(wl.mesh, wl.p, wl.a, dg_problem(wl), world)
        mine = _blocks_part(wl, part, rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        if rank == 0:
            union = {}
            for g in gathered:
                assert not (set(g) & set(union))
                union.update(g)
            ok = union == _blocks_full(wl)
            with open(os.path.join(out_dir, "ok"), "w") as f:
                f.write("1" if ok else "0")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_build_disjoint_parts(tmp_path):
    import torch.multiprocessing as mp

    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    assert (tmp_path / "ok").read_text() == "1"
