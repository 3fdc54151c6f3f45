"""Pipelined host-buffer assembly (dg_assemble_host_submit / _wait).

A sequence of assemblies on one mesh, with new coefficients a each time,
gives submission by submission bitwise the system that the synchronous
dg_assemble_host computes for the same inputs: the same kernels in the same
launch shape, whatever runs beside them.  Checked in FP32 and FP64, with the
waits one submission behind (the depth-2 pipeline a caller would run), all
at the end (the two device slots reused while earlier copies are queued),
and across a change of precision; a ticket that was never submitted is an
argument error.
"""
import numpy as np
import pytest

from paper_2007_04881_gb300 import configs, dg

from .helpers import dg_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda):
    import torch

    from paper_2007_04881_gb300 import build as B

    B.build()
    c = dg.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


@pytest.fixture(scope="module")
def wl():
    return configs.small2d(300, 5, 1, 4)


def coefficients(wl, k):
    rng = np.random.default_rng(1000 + k)
    return np.ascontiguousarray(wl.a * rng.uniform(0.5, 2.0, wl.ne))


def synchronous(m, prec, a):
    dt = np.float64 if prec == dg.DG_PREC_FP64 else np.float32
    vh, rh = np.zeros(m.nvals, dt), np.zeros(m.ndofs, dt)
    m.dg_assemble_host(prec, vh, rh, a=a)
    return vh, rh


def pinned_outputs(m, prec, k):
    import torch

    dt = torch.float64 if prec == dg.DG_PREC_FP64 else torch.float32
    return [(torch.zeros(m.nvals, dtype=dt).pin_memory(), torch.zeros(m.ndofs, dtype=dt).pin_memory())
            for _ in range(k)]


@pytest.mark.parametrize("prec", [dg.DG_PREC_FP32, dg.DG_PREC_FP64])
@pytest.mark.parametrize("lag", [1, 5])
def test_pipelined_equals_synchronous(ctx, wl, prec, lag):
    """lag 1: each wait one submission behind; lag 5: every wait after the
    last submission (each slot reused twice with copies still queued)."""
    import torch

    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    K = 5
    coef = [coefficients(wl, k) for k in range(K)]
    ref = [synchronous(m, prec, c) for c in coef]
    outs = pinned_outputs(m, prec, K)
    a_in = [torch.from_numpy(c).pin_memory() for c in coef]
    tickets = []
    for k in range(K):
        tickets.append(m.dg_assemble_host_submit(prec, outs[k][0], outs[k][1], a=a_in[k]))
        if k >= lag:
            m.dg_assemble_host_wait(tickets[k - lag])
    for t in tickets[max(0, K - lag):]:
        m.dg_assemble_host_wait(t)
    assert tickets == list(range(K))
    for k in range(K):
        assert np.array_equal(outs[k][0].numpy(), ref[k][0]), k
        assert np.array_equal(outs[k][1].numpy(), ref[k][1]), k
    # the coefficients differ, so the systems do
    assert not np.array_equal(ref[0][0], ref[1][0])


def test_precision_change_and_bad_ticket(ctx, wl):
    import torch

    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    with pytest.raises(dg.DGError):
        m.dg_assemble_host_wait(0)
    c0, c1 = coefficients(wl, 7), coefficients(wl, 8)
    o32 = pinned_outputs(m, dg.DG_PREC_FP32, 1)[0]
    o64 = pinned_outputs(m, dg.DG_PREC_FP64, 1)[0]
    t0 = m.dg_assemble_host_submit(dg.DG_PREC_FP32, o32[0], o32[1], a=torch.from_numpy(c0).pin_memory())
    t1 = m.dg_assemble_host_submit(dg.DG_PREC_FP64, o64[0], o64[1], a=torch.from_numpy(c1).pin_memory())
    m.dg_assemble_host_wait(t0)
    m.dg_assemble_host_wait(t1)
    r32, r64 = synchronous(m, dg.DG_PREC_FP32, c0), synchronous(m, dg.DG_PREC_FP64, c1)
    assert np.array_equal(o32[0].numpy(), r32[0]) and np.array_equal(o32[1].numpy(), r32[1])
    assert np.array_equal(o64[0].numpy(), r64[0]) and np.array_equal(o64[1].numpy(), r64[1])
    with pytest.raises(dg.DGError):
        m.dg_assemble_host_wait(t1 + 1)
