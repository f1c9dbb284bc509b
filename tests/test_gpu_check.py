"""The bounds-checked build (librepart_check.so, compiled with RP_CHECK): every
device gather index and every offset derived from the map or the sliced
layout is range-checked, and a violation is counted instead of trapping.

A child process loads that library (the binding holds one library per
process) and runs small parity cases over every kernel family -- map build,
value update (device and host buffers), FP64 / restarted / continued mixed
PCG on the sliced layout and on CSR, several parts (non-local entries and
halo gathers), the line preconditioner, BiCGStab FP64 and mixed, the adjoint
and the gradients, the batched kernel, the allocation-free SpMV -- against
the oracle with the tolerances of the other parity tests, then asserts that
no access was skipped. Two planted violations show that the checks fire; both
stay inside allocated memory even without the check (a CSR column past n into
a padded vector; a 4-bit slice index past its table, which reads the table
area's spare words).
"""
import multiprocessing as mp
import os
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _cases(q):
    sys.path[:0] = [ROOT, HERE]
    import torch

    from gpu_util import Case
    from oracle import repart_oracle as O
    from paper_2510_08536_gb300 import build, repart, synth
    out = {}
    try:
        path = build.build(check=True)
        repart.load(path)
        torch.cuda.set_device(0)
        dev = torch.device("cuda", 0)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
        repart.check_violations(reset=True)

        def solved(h, c, precision, tol=1e-9, **kw):
            x = torch.zeros(c.mesh.n_cells, dtype=torch.float64, device=dev)
            info = repart.solve(h, t(c.b), x, tol=tol, precision=precision, **kw)
            return info, x.cpu().numpy()

        # one part: map, update (device and pinned host buffers), three precisions,
        # sliced and CSR layouts, the line preconditioner
        c = Case((24, 20, 18), (2, 2, 2), sigma=1.0)
        ref = O.pcg(c.A, c.dinv, c.b, tol=1e-9)
        for layout in (repart.RP_LAYOUT_AUTO, repart.RP_LAYOUT_CSR):
            h = repart.build_repartition(c.mesh.ranks, layout=layout)
            m = repart.get_part_map(h, 0)
            for key in ("row_ptr", "col_idx", "src_of", "diag_pos"):
                assert np.array_equal(m[key].cpu().numpy(), getattr(c.map, key)), key
            repart.update_values_packed(h, torch.from_numpy(c.staging).pin_memory())
            assert np.array_equal(repart.get_values(h)["vals"].cpu().numpy(), c.vals)
            for prec in ("fp64", "mixed", "mixed_ru"):
                info, xs = solved(h, c, prec)
                assert info["status"] == 0 and c.true_rel_residual(xs) <= 1e-9, (layout, prec, info)
                bound = 1e-7 if prec == "fp64" else 1e-6
                assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= bound, (layout, prec)
            h.close()
        h = repart.build_repartition(c.mesh.ranks, precond=repart.RP_PRECOND_LINE)
        repart.update_values_packed(h, t(c.staging))
        for prec in ("fp64", "mixed_ru"):
            info, xs = solved(h, c, prec)
            assert info["status"] == 0 and c.true_rel_residual(xs) <= 1e-9, ("line", prec, info)
        h.close()
        out["one_part"] = True

        # several parts: local + non-local matrices, halo gathered from x
        for n_parts in (2, 8):
            h = repart.build_repartition(c.mesh.ranks, n_parts=n_parts)
            repart.update_values_packed(h, t(c.staging))
            for prec in ("fp64", "mixed_ru"):
                info, xs = solved(h, c, prec)
                assert info["status"] == 0 and c.true_rel_residual(xs) <= 1e-9, (n_parts, prec, info)
            h.close()
        out["parts"] = True

        # symmetric storage, adjoint and gradients (general storage with transpose positions)
        for symmetric in (True, False):
            cs = Case((14, 12, 10), (2, 2, 1), sigma=0.5, symmetric=symmetric)
            h = repart.build_repartition(cs.mesh.ranks, symmetric=symmetric, want_transpose=not symmetric)
            repart.update_values_packed(h, t(cs.staging))
            info, xs = solved(h, cs, "fp64")
            assert info["status"] == 0
            g = xs - synth.uniform_vector(cs.mesh, 1)
            lam = torch.zeros(cs.mesh.n_cells, dtype=torch.float64, device=dev)
            ainfo = repart.solve_adjoint(h, t(g), lam, tol=1e-12)
            assert ainfo["status"] == 0
            lref = np.linalg.solve(cs.A.toarray().T, g)
            assert np.linalg.norm(lam.cpu().numpy() - lref) / np.linalg.norm(lref) <= 1e-7
            gbuf = torch.zeros(h.n_slots, dtype=torch.float64, device=dev)
            repart.entry_grad(h, lam, t(xs), gbuf)
            ge = O.entry_grad(cs.map.row_ptr, cs.map.col_idx, lam.cpu().numpy(), xs)
            gs = O.slot_grad(cs.map.src_of, ge, h.n_slots)
            assert np.allclose(gbuf.cpu().numpy(), gs, rtol=1e-12, atol=1e-14)
            gf = torch.zeros(sum(r.n_faces + r.n_iface for r in cs.mesh.ranks), dtype=torch.float64, device=dev)
            repart.face_grad(h, lam, t(xs), gf)
            assert np.allclose(gf.cpu().numpy(), O.face_grad_ldu(cs.mesh.ranks, lam.cpu().numpy(), xs),
                               rtol=1e-12, atol=1e-14)
            h.close()
        out["adjoint"] = True

        # BiCGStab, FP64 and mixed, one part and several
        mesh = synth.box_mesh(20, 16, 12, 2, 2, 1)
        mstg = synth.momentum_staging(mesh, 0.5, 100)
        (mm,) = O.repartition_map(mesh.ranks, 1)
        Am = O.csr_matrix(mm.row_ptr, mm.col_idx, O.update_values(mm.src_of, mstg))
        b = synth.uniform_vector(mesh, 0)
        for n_parts in (1, 4):
            h = repart.build_repartition(mesh.ranks, n_parts=n_parts)
            repart.update_values_packed(h, t(mstg))
            for prec in ("fp64", "mixed"):
                x = torch.zeros(mesh.n_cells, dtype=torch.float64, device=dev)
                info = repart.solve_bicgstab(h, t(b), x, tol=1e-9, precision=prec)
                xs = x.cpu().numpy()
                assert info["status"] == 0 and np.linalg.norm(b - Am @ xs) / np.linalg.norm(b) <= 1e-9, (n_parts, prec)
            h.close()
        out["bicgstab"] = True

        # batched kernel: sliced and CSR, three precisions
        B = synth.Batch(count=9, lo=300, hi=3000, seed=5)
        bst, bb = B.staging(0.5, 100), B.rhs(0)
        ro = np.cumsum([0] + [m_.n_cells for m_ in B.meshes])
        so = np.cumsum([0] + [m_.staging_size() for m_ in B.meshes])
        for layout in (repart.RP_LAYOUT_AUTO, repart.RP_LAYOUT_CSR):
            h = repart.batch_build(B.systems, layout=layout)
            for prec in ("fp64", "mixed", "mixed_ru"):
                x = torch.zeros(B.n_rows, dtype=torch.float64, device=dev)
                infos = repart.batch_update_solve(h, t(bst), t(bb), x, 1e-9, prec)
                xs = x.cpu().numpy()
                for s_, rank in enumerate(B.systems):
                    xi, bi = xs[ro[s_]:ro[s_ + 1]], bb[ro[s_]:ro[s_ + 1]]
                    r = bi - O.ldu_matvec([rank], bst[so[s_]:so[s_ + 1]], xi)
                    assert infos[s_]["status"] == 0 and np.linalg.norm(r) / np.linalg.norm(bi) <= 1e-9, (layout, prec, s_)
            h.close()
        out["batch"] = True

        # allocation-free SpMV
        n = c.mesh.n_cells
        xv = t(synth.uniform_vector(c.mesh, 3))
        y = torch.empty(n, dtype=torch.float64, device=dev)
        repart.spmv_noalloc(n, t(c.map.row_ptr.astype(np.int32)), t(c.map.col_idx.astype(np.int32)), t(c.vals), xv, y)
        xh = xv.cpu().numpy()
        bound = 1e-14 * (abs(c.A) @ np.abs(xh)) + 1e-300  # summation order and FMA differ
        assert (np.abs(y.cpu().numpy() - c.A @ xh) <= bound).all()
        out["noalloc"] = True

        torch.cuda.synchronize()
        out["clean"] = repart.check_violations(reset=True)

        # planted 1: a CSR column past n (the vector is padded, so the unchecked read
        # would stay inside its allocation)
        nn = 64
        rp = torch.arange(nn + 1, dtype=torch.int32, device=dev)
        col = torch.arange(nn, dtype=torch.int32, device=dev)
        col[5] = nn + 6
        xp = torch.ones(2 * nn, dtype=torch.float64, device=dev)
        yp = torch.empty(nn, dtype=torch.float64, device=dev)
        repart.spmv_noalloc(nn, rp, col, torch.ones(nn, dtype=torch.float64, device=dev), xp, yp)
        out["planted_col"] = repart.check_violations(reset=True)
        out["planted_col_y5"] = float(yp[5])

        # planted 2: the first 4-bit index of slice 0, lane 0 set past its table (D < 16:
        # the shuffle would read a lane holding a spare zero word of the table area)
        h = repart.build_repartition(c.mesh.ranks)
        repart.update_values_packed(h, t(c.staging))
        sv = repart.SlicedView()
        repart._check(repart.load().rp_get_sliced_view(h.ptr, repart.ctypes.byref(sv)), "rp_get_sliced_view")
        tinfo0 = int(repart._view(sv.tinfo, 1, "<i4").cpu().numpy().view(np.uint32)[0])
        tabs = repart._view(sv.tabs, sv.tabs_len, "<i4").cpu().numpy()
        D = int(tabs[(tinfo0 & 0x7FFFFFFF) - 1])
        out["planted_D"] = (bool(tinfo0 >> 31), D)
        ibuf = repart._view(sv.ibuf, sv.ibuf_len, "<i4")  # device view of the handle's index words
        desc0 = repart._view(sv.desc, 2, "<i4").cpu().numpy()
        w = int(ibuf[int(desc0[1])].item()) & 0xFFFFFFFF
        ibuf[int(desc0[1])] = np.int32(np.uint32((w & ~0xF) | 0xF))
        xin = torch.ones(n, dtype=torch.float64, device=dev)
        yout = torch.empty(n, dtype=torch.float64, device=dev)
        repart.iter_spmv(h, xin, yout, "fp64")
        out["planted_index"] = repart.check_violations(reset=True)
        h.close()
    except Exception as exc:  # report to the parent
        import traceback
        out["error"] = traceback.format_exc()[-3000:]
    q.put(out)


def test_checked_build_parity_and_no_violations():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_cases, args=(q,))
    p.start()
    out = q.get(timeout=900)
    p.join(60)
    assert "error" not in out, out.get("error")
    assert p.exitcode == 0
    for key in ("one_part", "parts", "adjoint", "bicgstab", "batch", "noalloc"):
        assert out.get(key), key
    count, site, index = out["clean"]
    assert count == 0, f"{count} accesses skipped, first at site {site} index {index}"
    # the planted violations are caught at their sites (6: gathered row, 5: offset index)
    count, site, index = out["planted_col"]
    assert count == 1 and site == 6 and index == 64 + 6, out["planted_col"]
    assert out["planted_col_y5"] == 0.0  # the skipped product contributes nothing
    w4, D = out["planted_D"]
    assert w4 and D < 16
    count, site, index = out["planted_index"]
    assert count >= 1 and site == 5 and index == 15, out["planted_index"]
