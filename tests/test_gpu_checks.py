"""FP64 device checks of a whole representation (kerdock_check_reconstruction,
kerdock_check_tight_frame).

The checks are pinned first: on small padded cases their float64 results equal
a host float64 evaluation of the same identities (Lemma 6 read backwards;
Prop. 2's tight frame through the design) on the device representation, and a
planted error in one entry moves exactly the quantities it must.  Then they
check the benchmark's n = 1024 float32 representation and the precision
workload's n = 4096 representations (bfloat16, 68.75 GB; float32, 137.5 GB)
over every basis.

Tolerances.  Reconstruction: (1/d) sum_w |dR_w| <= max_w |dR_w|, so the error
is at most the largest entry error of the slab column: 10^-5 ||a_i|| for
float32 (the float32 FWHT is ~10^-6 relative), and for bfloat16
2^-9 (1/d) sum_w |R_w| <= 2^-9 ||a_i|| (round to nearest, 8 significant bits;
||R_b[:, i]|| = sqrt(d) ||a_i||) plus the tensor-core term TC_ABS[k] ||a_i||.  Tight frame: the residual relative to nb d |A A^T y|_inf is
bounded by twice the relative entry error (first order in dR): 10^-5 for
float32, 2^-8 for bfloat16 and 2 TC_ABS at d = 4096 with tensor-core stages.
"""
import numpy as np
import pytest

from gpu_common import TC_ABS, build_and_load, f32, okd, torch_cuda
import workloads

pytestmark = pytest.mark.gpu


def _host_checks(R, A64, k, Y, nb_all):
    """Float64 host evaluation on a (B, d, ldr) copy of the device representation."""
    B, d, ldr = R.shape
    m, n = A64.shape
    Apad = np.zeros((ldr, d))
    Apad[:m, :n] = A64
    signs = okd.sign_matrix(k)
    err = np.empty(B)
    for b in range(B):
        if b == d // 2:
            rec = R[b].T / np.sqrt(d)
        else:
            rec = okd.fwht_rows(R[b].T) / d * (1.0 - 2.0 * signs[b])[None, :]
        err[b] = np.abs(rec - Apad).max()
    rows = R.reshape(B * d, ldr)[:, :m]
    frame = ((rows @ Y.T)[:, :, None] * rows[:, None, :]).sum(axis=0)   # (P, m)
    ref = nb_all * d * (A64 @ (A64.T @ Y.T)).T
    return err, frame, ref


def _device_checks(plan, torch, Y):
    err = plan.check_reconstruction().cpu().numpy()
    frame, ref = plan.check_tight_frame(torch.from_numpy(Y).cuda())
    plan.sync()
    return err, frame.cpu().numpy(), ref.cpu().numpy()


@pytest.mark.parametrize("m,n,dtype", [(13, 16, "f32"), (13, 16, "bf16"), (40, 50, "f32"),
                                       (9, 64, "bf16")])
def test_checks_equal_host_fp64(m, n, dtype):
    torch = torch_cuda()
    K = build_and_load()
    rng = np.random.default_rng(m * n)
    A = rng.standard_normal((m, n)).astype(np.float32)
    A64 = f32(A)
    plan = K.KerdockPlan(m, n, J=4, K=2, S=4, dtype=dtype)
    plan.preprocess(torch.from_numpy(A).cuda())
    k = plan.info["k"]
    Y = rng.standard_normal((3, m))
    err, frame, ref = _device_checks(plan, torch, Y)
    R = plan.representation().float().cpu().numpy().astype(np.float64)
    herr, hframe, href = _host_checks(R, A64, k, Y, plan.info["num_bases"])
    np.testing.assert_allclose(err, herr, rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(ref, href, rtol=1e-12, atol=1e-12 * np.abs(href).max())
    np.testing.assert_allclose(frame, hframe, rtol=1e-10, atol=1e-10 * np.abs(hframe).max())
    # a sub-range of bases
    err2 = plan.check_reconstruction(1, 3).cpu().numpy()
    np.testing.assert_allclose(err2, herr[1:4], rtol=1e-9, atol=1e-14)
    plan.close()


def test_checks_detect_a_planted_error():
    torch = torch_cuda()
    K = build_and_load()
    n = 64
    A = workloads.random_orthogonal(n, 91).astype(np.float32)
    A64 = f32(A)
    plan = K.KerdockPlan(n, n, J=4, K=2, S=4)
    plan.preprocess(torch.from_numpy(A).cuda())
    Y = np.random.default_rng(92).standard_normal((2, n))
    err0, frame0, ref0 = _device_checks(plan, torch, Y)
    assert err0.max() < 1e-5
    b, w, i, delta = 7, 33, 5, 0.25
    rep = plan.representation()
    old = float(rep[b, w, i].item())
    rep[b, w, i] += delta
    torch.cuda.synchronize()
    err1, frame1, ref1 = _device_checks(plan, torch, Y)
    # column i of basis b comes back off by delta/d at every p; no other basis moves
    assert abs(err1[b] - delta / n) < 1e-5
    np.testing.assert_array_equal(np.delete(err1, b), np.delete(err0, b))
    # the frame moves by (R + delta e_i) <R + delta e_i, y> - R <R, y>
    row = rep[b, w, :n].double().cpu().numpy()
    row_old = row.copy()
    row_old[i] = old
    move = row[None, :] * (Y @ row)[:, None] - row_old[None, :] * (Y @ row_old)[:, None]
    np.testing.assert_allclose(frame1 - frame0, move, rtol=1e-6, atol=1e-6)
    np.testing.assert_array_equal(ref1, ref0)
    plan.close()


def _rel_frame_residual(frame, ref):
    return np.abs(frame - ref).max() / np.abs(ref).max()


def test_checks_n1024_f32_all_bases():
    torch = torch_cuda()
    K = build_and_load()
    wl = workloads.WORKLOADS["n1024"]
    A = wl.make_A().astype(np.float32)
    plan = K.KerdockPlan(wl.m, wl.n, J=wl.J, K=wl.K, S=wl.S)
    plan.preprocess(torch.from_numpy(A).cuda())
    Y = np.random.default_rng(93).standard_normal((4, wl.m))
    err, frame, ref = _device_checks(plan, torch, Y)
    a_max = np.linalg.norm(f32(A), axis=1).max()
    assert err.shape == (wl.n // 2 + 1,)
    assert err.max() <= 1e-5 * a_max, err.max()
    assert _rel_frame_residual(frame, ref) <= 1e-5
    np.testing.assert_allclose(ref, (513 * 1024) * (f32(A) @ (f32(A).T @ Y.T)).T, rtol=1e-10,
                               atol=1e-10 * np.abs(ref).max())
    plan.close()


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_checks_n4096_all_bases(dtype):
    torch = torch_cuda()
    K = build_and_load()
    wl = workloads.WORKLOADS["n4096_bf16"]
    A = wl.make_A().astype(np.float32)
    plan = K.KerdockPlan(wl.m, wl.n, J=wl.J, K=wl.K, S=wl.S, dtype=dtype)
    plan.preprocess(torch.from_numpy(A).cuda())
    Y = np.random.default_rng(94).standard_normal((4, wl.m))
    err, frame, ref = _device_checks(plan, torch, Y)
    a_max = np.linalg.norm(f32(A), axis=1).max()
    if dtype == "f32":
        rec_tol, frame_tol = 1e-5 * a_max, 1e-5
    else:
        rec_tol, frame_tol = (2.0 ** -9 + TC_ABS[12]) * a_max, 2 * TC_ABS[12]
    print(f"n=4096 {dtype}: reconstruction max {err.max():.3e} (bound {rec_tol:.3e}); "
          f"tight-frame relative residual {_rel_frame_residual(frame, ref):.3e}")
    assert err.max() <= rec_tol
    assert _rel_frame_residual(frame, ref) <= frame_tol
    plan.close()
    del plan
    torch.cuda.empty_cache()
