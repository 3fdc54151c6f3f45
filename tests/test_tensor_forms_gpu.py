"""Tensor-core forms of the local contractions (split-BF16 and 3xTF32, FP32
accumulation) against the FP64 oracle and the FP64 GPU form.

Tolerances (block max-norm relative, as the other parity tests):
  3xTF32: each operand x = hi + lo with TF32 halves keeps x to 2^-22
  relative and the dropped lo*lo term is below 2^-22 |uv|, so products are
  as accurate as FP32 products; the FP32 form's 5e-5 applies, and the
  whole-matrix relative Frobenius error is held to the 1e-6 target.
  split-BF16: bfloat16 halves keep x to 2^-18 and drop lo*lo below 2^-18
  |uv|: about 1e-5 relative per product, summed over up to ~10^3 rows with
  partial cancellation; 2e-4 per block and 2e-5 relative Frobenius.
  Load vectors: the same products, but each element's vector is dominated
  by the FP32 evaluation of the sin source near cancellation (3.4e-5 on the
  65k-cell mesh for FP32 and both tensor forms alike); 1e-4 per element.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_04881_gb300 import configs, dg

from .helpers import compare, dg_problem, oracle_blocks

pytestmark = pytest.mark.gpu

TOL = {dg.DG_PREC_TF32X3: 5e-5, dg.DG_PREC_BF16X3: 2e-4}
FRO = {dg.DG_PREC_TF32X3: 1e-6, dg.DG_PREC_BF16X3: 2e-5}
TOL_RHS = 1e-4
# on meshes where the FP32 basis values already limit the error (large
# degree-4 polyhedra), the bound is a multiple of the FP32 form's own error
REL32 = {dg.DG_PREC_TF32X3: 2.0, dg.DG_PREC_BF16X3: 20.0}
FORMS = [dg.DG_PREC_BF16X3, dg.DG_PREC_TF32X3]


@pytest.fixture(scope="module")
def ctx(cuda):
    import torch

    from paper_2007_04881_gb300 import build as B

    B.build()
    c = dg.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def run_gpu(ctx, wl, prec, how="fused", m=None):
    import torch

    m = m or dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    dt = torch.float64 if prec == dg.DG_PREC_FP64 else torch.float32
    vals = torch.full((m.nvals,), float("nan"), dtype=dt, device="cuda")
    r = torch.full((m.ndofs,), float("nan"), dtype=dt, device="cuda")
    if how == "split":
        m.dg_assemble_volume(prec, vals)
        m.dg_assemble_faces(prec, vals)
        m.dg_assemble_rhs(prec, r)
    else:
        m.dg_assemble(prec, vals, r)
    ctx.dg_sync()
    return m, vals.double().cpu().numpy(), r.double().cpu().numpy()


@pytest.mark.parametrize("prec", FORMS)
@pytest.mark.parametrize("which", ["2d", "3d"])
def test_against_oracle(ctx, prec, which):
    # every degree of the dimension, ragged tiles, advection and reaction on
    wl = configs.small2d(180, 7, 1, 6) if which == "2d" else configs.small3d(4, 10, 5, 1, 4)
    m, v, r = run_gpu(ctx, wl, prec)
    assert np.isfinite(v).all() and np.isfinite(r).all()
    om, ob = oracle_blocks(wl)
    ed, eo, er = compare(dg.to_blocks(m, v, r), om, ob, wl)
    print(f"\n{which} prec={prec}: diag {ed:.2e} off {eo:.2e} rhs {er:.2e}")
    assert ed < TOL[prec] and eo < TOL[prec] and er < TOL_RHS, (ed, eo, er)
    _, v64, _ = run_gpu(ctx, wl, dg.DG_PREC_FP64, m=m)
    _, v32, _ = run_gpu(ctx, wl, dg.DG_PREC_FP32, m=m)
    fro = np.linalg.norm(v - v64) / np.linalg.norm(v64)
    fro32 = np.linalg.norm(v32 - v64) / np.linalg.norm(v64)
    print(f"{which} prec={prec}: rel Frobenius vs FP64 {fro:.2e} (FP32 form {fro32:.2e})")
    # the tensor forms share the FP32 basis values and weights; only the
    # contraction arithmetic differs from the FP32 form
    assert fro < max(FRO[prec], REL32[prec] * fro32), (fro, fro32)


@pytest.mark.parametrize("prec", FORMS)
def test_adr2d_65k_sampled(ctx, prec):
    """Full-size 2D ADR workload in the benchmark's launch configuration:
    seeded sample of oracle blocks, whole-matrix error against FP64."""
    wl = configs.adr2d()
    m, v64, _ = run_gpu(ctx, wl, dg.DG_PREC_FP64)
    _, v, r = run_gpu(ctx, wl, prec, m=m)
    rng = np.random.default_rng(123)
    om = O.Mesh(wl.mesh)
    elems = np.sort(rng.choice(wl.ne, 300, replace=False))
    ifs = np.sort(rng.choice(om.ni, 300, replace=False))
    _, ob = oracle_blocks(wl, elems=elems, ifaces=ifs, om=om)
    ed, eo, er = compare(dg.to_blocks(m, v, r), om, ob, wl)
    fro = np.linalg.norm(v - v64) / np.linalg.norm(v64)
    print(f"\nadr2d_65k prec={prec}: diag {ed:.2e} off {eo:.2e} rhs {er:.2e} fro {fro:.2e}")
    assert ed < TOL[prec] and eo < TOL[prec] and er < TOL_RHS, (ed, eo, er)
    assert fro < FRO[prec], fro


@pytest.mark.parametrize("prec", FORMS)
def test_split_calls_and_determinism(ctx, prec):
    wl = configs.small2d(250, 13, 1, 5, b=(1.0, 0.5), c=1.0)
    m, v1, r1 = run_gpu(ctx, wl, prec)
    _, v2, r2 = run_gpu(ctx, wl, prec, m=m)
    assert np.array_equal(v1, v2) and np.array_equal(r1, r2)  # no atomics: bitwise
    _, v3, r3 = run_gpu(ctx, wl, prec, how="split", m=m)
    # the load vector alone takes the same products as in the fused pass
    assert np.array_equal(r1, r3)
    # volume then faces adds two FP32-rounded partial blocks
    assert np.abs(v1 - v3).max() <= 1e-5 * np.abs(v1).max()


@pytest.mark.parametrize("prec", FORMS)
def test_diffusion_only_3d(ctx, prec):
    """b = c = 0 skips the zero Phi rows of the volume points (load column only)."""
    wl = configs.small3d(4, 12, 8, 2, 3, b=(0.0, 0.0, 0.0), c=0.0)
    m, v, r = run_gpu(ctx, wl, prec)
    om, ob = oracle_blocks(wl)
    ed, eo, er = compare(dg.to_blocks(m, v, r), om, ob, wl)
    assert ed < TOL[prec] and eo < TOL[prec] and er < TOL_RHS, (ed, eo, er)


@pytest.mark.parametrize("prec", FORMS)
def test_learned_rules_in_tensor_forms(ctx, prec):
    """Elements with an installed 28-point learned rule take the same
    tensor-core contraction as the sub-triangle elements."""
    wl = configs.small2d(300, 45, 3, 3, b=(1.0, 0.5), c=1.0)
    m = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg_problem(wl))
    m.dg_quad_prepare()
    st = m.dg_quad_fit(None, iters=8, install=True)
    assert st["accepted"] > 0.8 * m.ne
    _, v64, r64 = run_gpu(ctx, wl, dg.DG_PREC_FP64, m=m)
    _, v, r = run_gpu(ctx, wl, prec, m=m)
    fro = np.linalg.norm(v - v64) / np.linalg.norm(v64)
    assert np.isfinite(v).all() and fro < FRO[prec], fro
    assert np.linalg.norm(r - r64) / np.linalg.norm(r64) < FRO[prec]
