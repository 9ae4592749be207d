"""Parity at the p-sweep sizes (about 20M DOFs per degree, the launch
configuration of `bench.py --sweep`), on sampled outputs the oracle computes
one by one:

* LOR rows (FP64 and FP32 values) computed alone from their sub-hexes;
* the high-order apply and the kappa-gradient kernel on sampled elements:
  every output of element e depends only on the elements around it, so the
  oracle runs on the 3x3x3 box of elements centred on e (clipped at the
  domain boundary) with x and gy set to 0 on the global boundary; the box's
  own Dirichlet treatment then only touches DOFs that are global boundary
  DOFs already (dirichlet=False for the apply, the oracle's backward masks
  the box boundary, which for e's DOFs is the global boundary).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2210_12253_gb300.inputs import boundary_mask, workload

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2210_12253_gb300.build import build
    build()


def box(prob, e, x, gy, ess):
    """Element box around e: (mesh, kappa, x_box, gy_box, local index of e's
    DOFs in the box, their global ids)."""
    p, q = prob.p, prob.q
    ne = (prob.nex, prob.ney, prob.nez)
    ec = (e % prob.nex, (e // prob.nex) % prob.ney, e // (prob.nex * prob.ney))
    lo = [max(0, c - 1) for c in ec]
    hi = [min(n - 1, c + 1) for c, n in zip(ec, ne)]
    bn = [h - l + 1 for l, h in zip(lo, hi)]
    # vertices of the box
    vid = []
    for c in range(lo[2], hi[2] + 2):
        for b in range(lo[1], hi[1] + 2):
            for a in range(lo[0], hi[0] + 2):
                vid.append(a + (ne[0] + 1) * (b + (ne[1] + 1) * c))
    V = prob.vertices.reshape(-1, 3)[vid]
    els = [ex + ne[0] * (ey + ne[1] * ez) for ez in range(lo[2], hi[2] + 1) for ey in range(lo[1], hi[1] + 1)
           for ex in range(lo[0], hi[0] + 1)]
    kap = prob.kappa[els]
    nx, ny = ne[0] * p + 1, ne[1] * p + 1
    bx, by, bz = (n * p + 1 for n in bn)
    gid = np.empty(bx * by * bz, np.int64)
    t = 0
    for K in range(bz):
        for J in range(by):
            for I in range(bx):
                gid[t] = (lo[0] * p + I) + nx * ((lo[1] * p + J) + ny * (lo[2] * p + K))
                t += 1
    xb = np.where(ess[gid], 0.0, x[gid])
    gb = np.where(ess[gid], 0.0, gy[gid])
    # local DOFs of e in the box
    oe = [c - l for c, l in zip(ec, lo)]
    loc = np.array([(oe[0] * p + i) + bx * ((oe[1] * p + j) + by * (oe[2] * p + k))
                    for k in range(p + 1) for j in range(p + 1) for i in range(p + 1)])
    return oracle.Mesh(*bn, V), kap, xb, gb, loc, gid[loc], els.index(e)


@pytest.mark.parametrize("p", range(2, 11))
def test_sweep_size_sampled_parity(p):
    from paper_2210_12253_gb300 import LOR
    prob = workload("c5_p%d" % p)
    q = p + 2
    op = LOR(p, prob.nex, prob.ney, prob.nez, torch.tensor(prob.vertices, device=DEV))
    op.set_coefficient(torch.tensor(prob.kappa.reshape(-1), device=DEV), check=True)
    assert 19.0e6 < op.ndof < 21.0e6
    mesh = oracle.Mesh(prob.nex, prob.ney, prob.nez, prob.vertices)
    rng = np.random.default_rng(100 + p)
    # ---- LOR rows, FP64 and FP32
    rp, _ = op.build_pattern()
    rows = np.unique(np.concatenate([rng.integers(0, op.ndof, 400), [0, op.ndof - 1, op.ndof // 2]]))
    cnt, cols, ref = oracle.lor_rows(mesh, p, q, prob.kappa, rows, True)
    rp_h = rp[torch.tensor(np.concatenate([rows, rows + 1]), device=DEV)].cpu().numpy()
    starts, ends = rp_h[:rows.size], rp_h[rows.size:]
    idx = torch.tensor(np.concatenate([np.arange(a, b) for a, b in zip(starts, ends)]), device=DEV)
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        vals = op.assemble(dtype)[idx].double().cpu().numpy()
        off = 0
        for k in range(rows.size):
            n = ends[k] - starts[k]
            assert n == cnt[k]
            r = ref[k, :n]
            assert np.abs(vals[off:off + n] - r).max() <= tol * np.abs(r).max(), (dtype, rows[k])
            off += n
        del vals
        torch.cuda.empty_cache()
    del rp
    # ---- apply and kappa gradient on sampled elements
    x = rng.standard_normal(op.ndof)
    gy = rng.standard_normal(op.ndof)
    ess = boundary_mask(prob.nex, prob.ney, prob.nez, p)
    y = op.apply(torch.tensor(x, device=DEV)).cpu().numpy()
    _, gk = op.apply_backward(torch.tensor(x, device=DEV), torch.tensor(gy, device=DEV), want_gx=False)
    gk = gk.reshape(op.nel, q ** 3)
    sample = np.unique(np.concatenate([rng.integers(0, op.nel, 6), [0, op.nel - 1]]))
    for e in sample:
        bm, kap, xb, gb, loc, gids, eb = box(prob, int(e), x, gy, ess)
        yb = oracle.ho_apply(bm, p, q, kap, xb, dirichlet=False)
        yref = np.where(ess[gids], x[gids], yb[loc])
        assert np.abs(y[gids] - yref).max() <= 1e-12 * np.abs(yb).max(), e
        _, gkb = oracle.ho_apply_backward(bm, p, q, kap, xb, gb, want_gx=False)
        g_gpu = gk[int(e)].cpu().numpy()
        assert np.abs(g_gpu - gkb[eb]).max() <= 1e-12 * np.abs(gkb[eb]).max(), e
    op.close()
