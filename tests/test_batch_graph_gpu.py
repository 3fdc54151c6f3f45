"""Batches of independent meshes in one pass, and recorded (CUDA-graph)
passes with the launch-shape autotuner."""
import numpy as np
import pytest

from paper_2007_04881_gb300 import configs, dg

from .helpers import compare, dg_problem, oracle_blocks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda):
    import torch

    from paper_2007_04881_gb300 import build as B

    B.build()
    c = dg.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def _members():
    out = []
    for k, (n, p) in enumerate([(60, 1), (150, 3), (40, 5), (95, 2), (120, 4), (33, 6)]):
        wl = configs.small2d(n, 50 + k, p, p, b=(1.0, 0.5), c=1.0)
        out.append(wl)
    return out


def _assemble(ctx, mesh, prec):
    import torch

    dt = torch.float64 if prec == dg.DG_PREC_FP64 else torch.float32
    v = torch.full((mesh.nvals,), float("nan"), dtype=dt, device="cuda")
    r = torch.full((mesh.ndofs,), float("nan"), dtype=dt, device="cuda")
    mesh.dg_assemble_step(prec, v, r)
    ctx.dg_sync()
    return v.double().cpu().numpy(), r.double().cpu().numpy()


@pytest.mark.parametrize("prec", [dg.DG_PREC_FP64, dg.DG_PREC_FP32])
def test_batch_equals_members(ctx, prec):
    members = _members()
    pb = dg_problem(members[0])
    bm = dg.Mesh(ctx, None, problem=pb, members=[(w.mesh, w.p, w.a) for w in members])
    eo, vo, do = bm.dg_batch_offsets()
    assert len(eo) == len(members) + 1
    vb, rb = _assemble(ctx, bm, prec)
    for k, w in enumerate(members):
        m = dg.Mesh(ctx, w.mesh, w.p, w.a, pb)
        v, r = _assemble(ctx, m, prec)
        assert vo[k + 1] - vo[k] == m.nvals and do[k + 1] - do[k] == m.ndofs
        # the same element computations, grouped differently: bitwise equal
        assert np.array_equal(vb[vo[k]:vo[k + 1]], v)
        assert np.array_equal(rb[do[k]:do[k + 1]], r)


def test_batch_member_vs_oracle(ctx):
    members = _members()
    pb = dg_problem(members[0])
    bm = dg.Mesh(ctx, None, problem=pb, members=[(w.mesh, w.p, w.a) for w in members])
    eo, vo, do = bm.dg_batch_offsets()
    vb, rb = _assemble(ctx, bm, dg.DG_PREC_FP64)
    k = 2
    w = members[k]
    m = dg.Mesh(ctx, w.mesh, w.p, w.a, pb)
    got = dg.to_blocks(m, vb[vo[k]:vo[k + 1]], rb[do[k]:do[k + 1]])
    om, ob = oracle_blocks(w)
    ed, eo_, er = compare(got, om, ob, w)
    assert max(ed, eo_, er) < 1e-12


@pytest.mark.parametrize("autotune", [False, True])
def test_graph_replay_equals_direct(ctx, autotune):
    import torch

    w = configs.small2d(400, 77, 1, 5)
    m = dg.Mesh(ctx, w.mesh, w.p, w.a, dg_problem(w))
    v_ref, r_ref = _assemble(ctx, m, dg.DG_PREC_FP32)
    v = torch.zeros(m.nvals, dtype=torch.float32, device="cuda")
    r = torch.zeros(m.ndofs, dtype=torch.float32, device="cuda")
    g = m.dg_graph_create(dg.DG_PREC_FP32, v, r, autotune=autotune)
    info = g.dg_graph_info()
    assert info["launches"] >= 3 + 5
    for _ in range(3):
        v.zero_()
        g.dg_graph_launch()
        ctx.dg_sync()
        assert np.array_equal(v.double().cpu().numpy(), v_ref)
        assert np.array_equal(r.double().cpu().numpy(), r_ref)
    g.close()


@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("prec", [dg.DG_PREC_FP64, dg.DG_PREC_FP32])
def test_assemble_batch_equals_member_steps(ctx, prec, use_graph):
    """dg_assemble_batch over separately uploaded meshes (direct or recorded)
    writes each member's buffers bit for bit as its own dg_assemble_step."""
    import torch

    members = _members()
    pb = dg_problem(members[0])
    meshes = [dg.Mesh(ctx, w.mesh, w.p, w.a, pb) for w in members]
    dt = torch.float64 if prec == dg.DG_PREC_FP64 else torch.float32
    vals = [torch.full((m.nvals,), float("nan"), dtype=dt, device="cuda") for m in meshes]
    rhs = [torch.full((m.ndofs,), float("nan"), dtype=dt, device="cuda") for m in meshes]
    rhs[3] = None  # a member without a load vector
    for _ in range(2):  # twice: the second call overwrites the first
        dg.dg_assemble_batch(ctx, meshes, prec, vals, rhs, use_graph=use_graph)
        ctx.dg_sync()
    for k, m in enumerate(meshes):
        v, r = _assemble(ctx, m, prec)
        assert np.array_equal(vals[k].double().cpu().numpy(), v), k
        if rhs[k] is not None:
            assert np.array_equal(rhs[k].double().cpu().numpy(), r), k


@pytest.mark.parametrize("dim", [2, 3])
def test_tile_variants_bitwise_equal(ctx, dim):
    """Every register-tile variant of the FP32 row kernels (the autotuner's
    candidates) sums each entry over the same points in the same order: the
    matrix and load vector are bitwise those of the default tiles, on the
    moment and on the per-point volume path."""
    import torch

    if dim == 2:
        w = configs.small2d(500, 91, 1, 6, b=(1.0, 0.5), c=1.0)
    else:
        w = configs.small3d(6, 20, 92, 2, 3)
    m = dg.Mesh(ctx, w.mesh, w.p, w.a, dg_problem(w))
    try:
        for path in (1, 0):
            ctx.dg_set_volume_path(path)
            ctx.dg_set_tile_variants(None)
            v0, r0 = _assemble(ctx, m, dg.DG_PREC_FP32)
            for var in (1, 2):
                ctx.dg_set_tile_variants([var] * 9)
                v, r = _assemble(ctx, m, dg.DG_PREC_FP32)
                assert np.array_equal(v, v0), (path, var)
                assert np.array_equal(r, r0), (path, var)
    finally:
        ctx.dg_set_volume_path(1)
        ctx.dg_set_tile_variants(None)


def test_autotuner_records_tiles(ctx):
    import torch

    w = configs.small2d(600, 93, 1, 5, b=(1.0, 0.5), c=1.0)
    m = dg.Mesh(ctx, w.mesh, w.p, w.a, dg_problem(w))
    v = torch.zeros(m.nvals, dtype=torch.float32, device="cuda")
    r = torch.zeros(m.ndofs, dtype=torch.float32, device="cuda")
    g = m.dg_graph_create(dg.DG_PREC_FP32, v, r, autotune=True)
    info = g.dg_graph_info()
    present = sorted(set(int(q) for q in w.p))
    assert sorted(int(k[1:]) for k in info["tile_tm"]) == present
    assert info["tile_tm"]["p4"] in (8, 5, 4) and info["tile_tm"]["p3"] in (5, 4)
    assert info["tuner_trials"] >= 12 + 1 + 2 + 2
    # the reference: the direct pass on the volume path and pass the tuner
    # chose (tile variants do not change the bits; the paths do)
    path = {"per-point": 0, "moments": 1, "exact-moments": 2}[info["volume_path"]]
    ctx.dg_set_volume_path(path)
    ctx.dg_set_persistent(info["persistent"])
    try:
        v_ref, r_ref = _assemble(ctx, m, dg.DG_PREC_FP32)
    finally:
        ctx.dg_set_volume_path(1)
        ctx.dg_set_persistent(False)
    g.dg_graph_launch()
    ctx.dg_sync()
    assert np.array_equal(v.double().cpu().numpy(), v_ref)
    assert np.array_equal(r.double().cpu().numpy(), r_ref)
    g.close()


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_group_split_bitwise(ctx, which):
    """Degree groups in parts on their own streams: every element is computed
    by the same kernel, so the system is bitwise that of whole groups."""
    if which == "2d":
        w = configs.small2d(700, 95, 1, 5, b=(1.0, 0.5), c=1.0)
    else:
        w = configs.small3d(6, 60, 96, 3, 3)  # one degree group: parts alone make it concurrent
    m = dg.Mesh(ctx, w.mesh, w.p, w.a, dg_problem(w))
    v0, r0 = _assemble(ctx, m, dg.DG_PREC_FP32)
    try:
        for split in ([1, 2, 3, 4, 2, 3, 1, 1, 1], [1, 4, 4, 4, 4, 4, 4, 1, 1]):
            ctx.dg_set_group_split(split)
            v, r = _assemble(ctx, m, dg.DG_PREC_FP32)
            assert np.array_equal(v, v0) and np.array_equal(r, r0), split
        with pytest.raises(dg.DGError):
            ctx.dg_set_group_split([1, 5, 1, 1, 1, 1, 1, 1, 1])
    finally:
        ctx.dg_set_group_split(None)
