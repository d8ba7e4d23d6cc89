"""GPU parity: the CUDA library against the FP64 oracle, through the C ABI.

Tolerances: per-entry matrix values within one FP32 rounding of the FP64
oracle (plus 1e-11 for the two independent FP64 geometries); per FP32 SpMV
rel L2 <= 1e-5; per reconstruction rel L2 <= 1e-3 (the targets of the
method's hot path).  Inputs are seeded synthetic phantoms.
"""

import functools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import radon, tv
from paper_1705_07497_gb300 import ct, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPMV_TOL = 1e-5
RECON_TOL = 1e-3


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


@functools.lru_cache(maxsize=None)
def oracle_A(n, nt, keep, nb):
    return radon.siddon_matrix(n, nt, keep, nb)


@functools.lru_cache(maxsize=None)
def gpu_A(n, nt, keep, nb, flags=0):
    return ct.Matrix(n, nt, keep, nb, flags)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def t32(x, dev):
    return torch.tensor(np.asarray(x), dtype=torch.float32, device=dev)


GEOMS = [
    (64, 90, 3, 91),    # the 64x64 workload: rays on pixel edges at 0 and pi/2
    (16, 12, 1, 23),
    (15, 17, 2, 22),    # odd N, even bin count
    (33, 37, 2, 47),
    (1, 4, 1, 2),       # one pixel
    (40, 7, 1, 100),    # many empty rows (bins beyond the image)
]


def _compare_csr(rp, ci, va, ref):
    """|gpu - oracle| <= 2^-24 |oracle| + 1e-11 on the union of both patterns
    (so an entry missing on either side must itself be below 1e-11), and
    strictly increasing columns in every row."""
    ref = sp.csr_matrix(ref)
    got = sp.csr_matrix((va.astype(np.float64), ci, rp), shape=ref.shape)
    for r in range(ref.shape[0]):
        assert np.all(np.diff(ci[rp[r]:rp[r + 1]]) > 0)
    diff = (got - ref).tocoo()
    ref_at = np.asarray(ref[diff.row, diff.col]).ravel()
    assert np.all(np.abs(diff.data) <= 2.0 ** -24 * np.abs(ref_at) + 1e-11)


@pytest.mark.parametrize("geom", GEOMS)
def test_matrix_entries_match_oracle(dev, geom):
    ref = oracle_A(*geom)
    M = gpu_A(*geom)
    assert (M.rows, M.cols) == ref.shape
    assert M.nnz == ref.nnz
    rp, ci, va = M.export(0)
    _compare_csr(rp, ci, va, ref)
    # A^T holds exactly the transpose (bit for bit)
    trp, tci, tva = M.export(1)
    got = sp.csr_matrix((va, ci, rp), shape=ref.shape)
    gotT = sp.csr_matrix((tva, tci, trp), shape=(ref.shape[1], ref.shape[0]))
    assert (got.T.tocsr() != gotT).nnz == 0


def test_matrix_entries_full_size_sampled(dev):
    geom = (512, 720, 4, 725)
    ref = oracle_A(*geom)
    M = gpu_A(*geom)
    assert M.nnz == ref.nnz == 60599464
    rp, ci, va = M.export(0)
    rows = np.random.Generator(np.random.PCG64(7)).choice(ref.shape[0], 2000, replace=False)
    for r in rows:
        a, b = ref.indptr[r], ref.indptr[r + 1]
        np.testing.assert_array_equal(ci[rp[r]:rp[r + 1]], ref.indices[a:b])
        d = np.abs(va[rp[r]:rp[r + 1]].astype(np.float64) - ref.data[a:b])
        assert np.all(d <= 2.0 ** -24 * ref.data[a:b] + 1e-11)


@pytest.mark.parametrize("geom", GEOMS[:4] + [(256, 360, 2, 363)])
@pytest.mark.parametrize("batch", [1, 3, 40, 64, 65])
def test_forward_adjoint_parity(dev, geom, batch):
    ref = oracle_A(*geom)
    M = gpu_A(*geom)
    x = inputs.random_vector(ref.shape[1] * batch, 21).reshape(ref.shape[1], batch)
    y = inputs.random_vector(ref.shape[0] * batch, 22).reshape(ref.shape[0], batch)
    yg = torch.empty((ref.shape[0], batch), dtype=torch.float32, device=dev)
    xg = torch.empty((ref.shape[1], batch), dtype=torch.float32, device=dev)
    M.forward(t32(x, dev), yg)
    M.adjoint(t32(y, dev), xg)
    assert rel(yg.cpu().numpy(), ref @ x) <= SPMV_TOL
    assert rel(xg.cpu().numpy(), ref.T @ y) <= SPMV_TOL


def test_forward_adjoint_host_buffers(dev):
    geom = (64, 90, 3, 91)
    ref = oracle_A(*geom)
    M = gpu_A(*geom)
    x = inputs.random_vector(ref.shape[1], 23).astype(np.float32)
    y = np.zeros(ref.shape[0], dtype=np.float32)
    M.forward(x, y)
    assert rel(y, ref @ x.astype(np.float64)) <= SPMV_TOL
    xb = np.zeros(ref.shape[1], dtype=np.float32)
    M.adjoint(y, xb)
    assert rel(xb, ref.T @ y.astype(np.float64)) <= SPMV_TOL


def test_adjoint_identity_on_gpu(dev):
    geom = (256, 360, 2, 363)
    M = gpu_A(*geom)
    x = t32(inputs.random_vector(M.cols, 24), dev)
    y = t32(inputs.random_vector(M.rows, 25), dev)
    Ax = torch.empty(M.rows, device=dev)
    Aty = torch.empty(M.cols, device=dev)
    M.forward(x, Ax)
    M.adjoint(y, Aty)
    lhs = float((Ax.double() * y.double()).sum())
    rhs = float((x.double() * Aty.double()).sum())
    scale = float((Ax.double().abs() * y.double().abs()).sum())
    assert abs(lhs - rhs) <= 1e-6 * scale


def test_forward_full_size_sampled_rows(dev):
    """512x512, 180 of 720 angles, 725 bins: sampled rows of y = A x recomputed
    one by one by the oracle."""
    geom = (512, 720, 4, 725)
    ref = oracle_A(*geom)
    M = gpu_A(*geom)
    x = inputs.ellipse_phantom(512, 1000).ravel()
    yg = torch.empty(M.rows, device=dev)
    M.forward(t32(x, dev), yg)
    y = yg.cpu().numpy()
    rows = np.random.Generator(np.random.PCG64(8)).choice(M.rows, 3000, replace=False)
    want = np.array([ref.data[ref.indptr[r]:ref.indptr[r + 1]] @ x[ref.indices[ref.indptr[r]:ref.indptr[r + 1]]]
                     for r in rows])
    scale = np.abs(want).max()
    assert np.abs(y[rows] - want).max() <= 1e-5 * scale
    # adjoint: sampled pixels
    yv = inputs.random_vector(M.rows, 26)
    xg = torch.empty(M.cols, device=dev)
    M.adjoint(t32(yv, dev), xg)
    At = ref.T.tocsr()
    pix = np.random.Generator(np.random.PCG64(9)).choice(M.cols, 3000, replace=False)
    want = np.array([At.data[At.indptr[p]:At.indptr[p + 1]] @ yv[At.indices[At.indptr[p]:At.indptr[p + 1]]]
                     for p in pix])
    got = xg.cpu().numpy()[pix]
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()


CG_CASES = {
    "split_bregman": (0.0, 1.0, 0.1),
    "resolvent": (1.0, 0.05, 0.0),
    "normal_eq": (0.0, 1.0, 1.0),
    "gradient_only": (1.0, 0.0, 0.5),
}


@pytest.mark.parametrize("case", sorted(CG_CASES))
def test_cg_solve_parity(dev, case):
    c_id, c_ata, c_grad = CG_CASES[case]
    geom = (64, 90, 3, 91)
    n = geom[0]
    ref = oracle_A(*geom)
    M = gpu_A(*geom)
    rhs = inputs.random_vector(n * n, 31)
    u0 = inputs.random_vector(n * n, 32) * 0.1
    op = tv.make_operator(ref, (n, n), c_id, c_ata, c_grad)
    want, st = tv.cg(op, rhs, u0, 10)
    u = t32(u0, dev)
    s = M.cg_solve(t32(rhs, dev), u, c_id, c_ata, c_grad, 10)
    assert s["status"] == 0 and s["iters"] == st["iters"] == 10
    assert rel(u.cpu().numpy(), want) <= 1e-4
    assert abs(s["final_rel_res"] - st["rel_res"]) <= 1e-3 * st["rel_res"] + 1e-7


def test_cg_tolerance_stop_matches_oracle(dev):
    geom = (64, 90, 3, 91)
    n = geom[0]
    ref = oracle_A(*geom)
    M = gpu_A(*geom)
    rhs = inputs.random_vector(n * n, 33)
    op = tv.make_operator(ref, (n, n), 1.0, 0.02, 0.0)
    want, st = tv.cg(op, rhs, np.zeros(n * n), 200, rel_tol=1e-4)
    u = torch.zeros(n * n, device=dev)
    s = M.cg_solve(t32(rhs, dev), u, 1.0, 0.02, 0.0, 200, rel_tol=1e-4)
    assert st["iters"] < 200
    assert abs(s["iters"] - st["iters"]) <= 1
    assert s["final_rel_res"] <= 1e-4
    assert rel(u.cpu().numpy(), want) <= 1e-3


def _sb_case(geom, seed, noise=None):
    n = geom[0]
    ref = oracle_A(*geom)
    truth = inputs.ellipse_phantom(n, seed)
    f = ref @ truth.ravel()
    if noise:
        f = inputs.gaussian_noisy(f, noise, seed + 1)
    return ref, truth, f


def test_split_bregman_64_workload(dev):
    """64x64, 30 of 90 angles, 91 bins, no noise, alpha 1, lambda 0.1, 20 x 10."""
    geom = (64, 90, 3, 91)
    ref, truth, f = _sb_case(geom, 0)
    M = gpu_A(*geom)
    want = tv.split_bregman(ref, f, (64, 64), 1.0, 0.1, 20, 10)
    u = torch.zeros(64 * 64, device=dev)
    st = M.split_bregman(t32(f, dev), u, 1.0, 0.1, 20, 10)
    assert st["status"] == 0 and st["outer_done"] == 20
    assert rel(u.cpu().numpy(), want["u"].ravel()) <= RECON_TOL
    assert abs(st["first_update_l1"] - want["updates"][0]) <= 1e-3 * want["updates"][0]
    assert abs(st["last_update_l1"] - want["updates"][-1]) <= 1e-2 * want["updates"][-1]


def test_split_bregman_host_buffers(dev):
    geom = (64, 90, 3, 91)
    ref, truth, f = _sb_case(geom, 0)
    M = gpu_A(*geom)
    want = tv.split_bregman(ref, f, (64, 64), 1.0, 0.1, 5, 10)["u"].ravel()
    u = np.zeros(64 * 64, dtype=np.float32)
    st = M.split_bregman(f.astype(np.float32), u, 1.0, 0.1, 5, 10)
    assert st["outer_done"] == 5
    assert rel(u, want) <= RECON_TOL


def test_split_bregman_512_first_update(dev):
    """512x512, 180 of 720 angles, 725 bins, 1% Gaussian noise, alpha = lambda = 1,
    one Bregman update of 20 CG steps against the oracle.  The first update is
    well conditioned (FP64 perturbations of A at 1e-9 move it by 1e-5); later
    updates of this workload amplify FP64 rounding itself to ~1e-3, see
    test_split_bregman_512_band."""
    geom = (512, 720, 4, 725)
    ref, truth, f = _sb_case(geom, 1000, noise=0.01)
    M = gpu_A(*geom)
    want = tv.split_bregman(ref, f, (512, 512), 1.0, 1.0, 1, 20)
    u = torch.zeros(512 * 512, device=dev)
    st = M.split_bregman(t32(f, dev), u, 1.0, 1.0, 1, 20)
    assert st["outer_done"] == 1
    assert rel(u.cpu().numpy(), want["u"].ravel()) <= 1e-4
    assert abs(st["first_update_l1"] - want["updates"][0]) <= 1e-4 * want["updates"][0]


def test_split_bregman_stop_rule(dev):
    geom = (64, 90, 3, 91)
    ref, truth, f = _sb_case(geom, 0)
    M = gpu_A(*geom)
    want = tv.split_bregman(ref, f, (64, 64), 1.0, 0.1, 200, 10, stop_rel_update=0.05)
    u = torch.zeros(64 * 64, device=dev)
    st = M.split_bregman(t32(f, dev), u, 1.0, 0.1, 200, 10, stop_rel_update=0.05)
    assert want["outer_done"] < 200
    assert abs(st["outer_done"] - want["outer_done"]) <= 1
    if st["outer_done"] == want["outer_done"]:
        assert rel(u.cpu().numpy(), want["u"].ravel()) <= RECON_TOL


@pytest.mark.parametrize("r,square", [(1, False), (3, False), (2, True)])
def test_surrogate_stencil_matches_oracle(dev, r, square):
    geom = (64, 90, 3, 91)
    ref = oracle_A(*geom)
    M = gpu_A(*geom)
    want = tv.surrogate_stencil(tv.point_response(ref, 64), r, "square" if square else "disc")
    got = M.surrogate_stencil(r, square)
    assert set(got) == set(want)
    for k, v in want.items():
        assert abs(got[k] - v) <= 1e-12 * abs(want[(0, 0)])


@pytest.mark.parametrize("r", [1, 3])
def test_surrogate_split_bregman_parity(dev, r):
    """Eq. surr_SBupd: the surrogate T replaces A^T A, the rhs keeps alpha A^T f."""
    geom = (64, 90, 3, 91)
    ref, truth, f = _sb_case(geom, 0)
    M = gpu_A(*geom)
    taps = tv.surrogate_stencil(tv.point_response(ref, 64), r, "disc")
    T = tv.surrogate_matrix(taps, 64)
    want = tv.split_bregman(ref, f, (64, 64), 1.0, 1.0, 20, 10, normal=lambda x: T @ x)
    u = torch.zeros(64 * 64, device=dev)
    st = M.split_bregman(t32(f, dev), u, 1.0, 1.0, 20, 10, surrogate_r=r)
    assert st["status"] == 0
    assert rel(u.cpu().numpy(), want["u"].ravel()) <= RECON_TOL


def test_surrogate_indefinite_window_reports_breakdown(dev):
    """The 5x5 square window of this geometry gives an indefinite alpha T +
    lambda grad^T grad: the oracle's CG breaks down, and so must the library's
    (reported as a status, not hidden)."""
    geom = (64, 90, 3, 91)
    ref, truth, f = _sb_case(geom, 0)
    M = gpu_A(*geom)
    taps = tv.surrogate_stencil(tv.point_response(ref, 64), 2, "square")
    T = tv.surrogate_matrix(taps, 64)
    with pytest.raises(tv.Breakdown):
        tv.split_bregman(ref, f, (64, 64), 1.0, 1.0, 20, 10, normal=lambda x: T @ x)
    u = torch.zeros(64 * 64, device=dev)
    with pytest.raises(ct.CtError) as ei:
        M.split_bregman(t32(f, dev), u, 1.0, 1.0, 20, 10, surrogate_r=2, square=True)
    assert ei.value.code == ct.CT_ERR_BREAKDOWN


def test_nonfinite_rhs_is_reported(dev):
    geom = (16, 12, 1, 23)
    M = gpu_A(*geom)
    rhs = torch.ones(M.cols, device=dev)
    rhs[5] = float("nan")
    u = torch.zeros(M.cols, device=dev)
    with pytest.raises(ct.CtError) as ei:
        M.cg_solve(rhs, u, 0.0, 1.0, 1.0, 5)
    assert ei.value.code == ct.CT_ERR_NONFINITE


def test_indefinite_operator_reports_breakdown(dev):
    geom = (16, 12, 1, 23)
    M = gpu_A(*geom)
    rhs = t32(inputs.random_vector(M.cols, 34), dev)
    u = torch.zeros(M.cols, device=dev)
    with pytest.raises(ct.CtError) as ei:
        M.cg_solve(rhs, u, -1.0, 0.0, 0.0, 5)
    assert ei.value.code == ct.CT_ERR_BREAKDOWN
    # the handle stays usable afterwards
    s = M.cg_solve(rhs, u, 1.0, 0.0, 0.0, 5)
    assert s["status"] == 0


def test_zero_iterations_and_zero_rhs(dev):
    geom = (16, 12, 1, 23)
    M = gpu_A(*geom)
    u0 = t32(inputs.random_vector(M.cols, 35), dev)
    u = u0.clone()
    s = M.cg_solve(torch.zeros(M.cols, device=dev), u, 0.0, 1.0, 1.0, 0)
    assert s["iters"] == 0 and torch.equal(u, u0)
    u = torch.zeros(M.cols, device=dev)
    s = M.cg_solve(torch.zeros(M.cols, device=dev), u, 0.0, 1.0, 1.0, 7)
    assert s["iters"] == 0 and s["status"] == 0 and float(u.abs().max()) == 0.0


def test_surrogate_warm_start_then_exact(dev):
    """Sec. 5's warm-start strategy: surrogate-T updates, then exact updates
    started from that reconstruction (initial guess only), against the oracle
    doing the same."""
    geom = (64, 90, 3, 91)
    A = radon.siddon_matrix(*geom)
    M = ct.Matrix(*geom)
    f = A @ inputs.ellipse_phantom(64, 21).ravel()
    T = tv.surrogate_matrix(tv.surrogate_stencil(tv.point_response(A, 64), 3), 64)
    u1 = tv.split_bregman(A, f, (64, 64), 1.0, 0.1, 8, 10, normal=lambda x: T @ x)["u"]
    want = tv.split_bregman(A, f, (64, 64), 1.0, 0.1, 6, 10, u0=u1.ravel())["u"].ravel()
    u = torch.zeros(64 * 64, dtype=torch.float32, device=dev)
    ft = torch.tensor(f, dtype=torch.float32, device=dev)
    M.split_bregman(ft, u, 1.0, 0.1, 8, 10, surrogate_r=3)
    M.split_bregman(ft, u, 1.0, 0.1, 6, 10)
    got = u.cpu().double().numpy()
    assert np.linalg.norm(got - want) <= 1e-3 * np.linalg.norm(want)


def test_many_angles_stage_the_band_in_chunks(dev):
    """400 kept angles: a tile's band (about 8,800 slots) is staged in three
    angle chunks by the adjoint kernels.  Products, CG and split Bregman
    against the oracle."""
    geom = (64, 400, 1, 91)
    ref = oracle_A(*geom)
    M = gpu_A(*geom)
    x = inputs.random_vector(ref.shape[1], 61)
    y = inputs.random_vector(ref.shape[0], 62)
    yg = torch.empty(ref.shape[0], device=dev)
    xg = torch.empty(ref.shape[1], device=dev)
    M.forward(t32(x, dev), yg)
    M.adjoint(t32(y, dev), xg)
    assert rel(yg.cpu().numpy(), ref @ x) <= SPMV_TOL
    assert rel(xg.cpu().numpy(), ref.T @ y) <= SPMV_TOL
    op = tv.make_operator(ref, (64, 64), 0.0, 1.0, 0.5)
    rhs = inputs.random_vector(ref.shape[1], 63)
    u = torch.zeros(ref.shape[1], device=dev)
    M.cg_solve(t32(rhs, dev), u, 0.0, 1.0, 0.5, 10)
    want, _ = tv.cg(op, rhs, np.zeros(ref.shape[1]), 10)
    assert rel(u.cpu().numpy(), want) <= 1e-4
    f = ref @ inputs.ellipse_phantom(64, 64).ravel()
    u = torch.zeros(ref.shape[1], device=dev)
    M.split_bregman(t32(f, dev), u, 1.0, 0.5, 8, 10)
    want = tv.split_bregman(ref, f, (64, 64), 1.0, 0.5, 8, 10)["u"].ravel()
    assert rel(u.cpu().numpy(), want) <= 1e-3


@pytest.mark.parametrize("host", [False, True])
def test_chambolle_pock_matches_oracle(dev, host):
    """Chambolle-Pock with the resolvent of Eq. PD_resolve solved by 10 CG
    steps per update, 20 updates, against the oracle; device and host pointers."""
    geom = (64, 90, 3, 91)
    A = oracle_A(*geom)
    M = gpu_A(*geom)
    f = inputs.gaussian_noisy(A @ inputs.ellipse_phantom(64, 31).ravel(), 0.01, 32)
    step = 0.99 / np.sqrt(8.0)
    want = tv.chambolle_pock(A, f, (64, 64), 1.0, step, step, 20, 10)
    if host:
        u = np.zeros(64 * 64, dtype=np.float32)
        st = M.chambolle_pock(f.astype(np.float32), u, 1.0, step, step, 20, 10)
        got = u.astype(np.float64)
    else:
        u = torch.zeros(64 * 64, dtype=torch.float32, device=dev)
        st = M.chambolle_pock(t32(f, dev), u, 1.0, step, step, 20, 10)
        got = u.cpu().double().numpy()
    assert st["status"] == 0 and st["outer_done"] == 20
    assert rel(got, want["u"].ravel()) <= 1e-4
    assert abs(st["first_update_l1"] - want["updates"][0]) <= 1e-4 * want["updates"][0]


def test_chambolle_pock_warm_start_and_batch_limit(dev):
    geom = (64, 90, 3, 91)
    A = oracle_A(*geom)
    M = gpu_A(*geom)
    f = A @ inputs.ellipse_phantom(64, 33).ravel()
    u0 = inputs.ellipse_phantom(64, 34).ravel()
    want = tv.chambolle_pock(A, f, (64, 64), 0.5, 0.3, 0.3, 6, 8, theta=0.5, u0=u0)
    u = t32(u0, dev)
    M.chambolle_pock(t32(f, dev), u, 0.5, 0.3, 0.3, 6, 8, theta=0.5)
    assert rel(u.cpu().numpy(), want["u"].ravel()) <= 1e-4
    with pytest.raises(ct.CtError) as e:
        M.chambolle_pock(torch.zeros((M.rows, 2), device=dev), torch.zeros((M.cols, 2), device=dev),
                         1.0, 0.3, 0.3, 3, 3)
    assert e.value.code == ct.CT_ERR_UNSUPPORTED


def test_batched_products_from_an_offset_view(dev):
    """A batch of 64 from an array that starts 4 bytes into its allocation: the
    products must not assume the alignment paired-slice loads need."""
    geom = (64, 90, 3, 91)
    ref = oracle_A(*geom)
    M = gpu_A(*geom)
    B = 64
    y = inputs.random_vector(ref.shape[0] * B, 64).reshape(ref.shape[0], B)
    big = torch.empty(ref.shape[0] * B + 1, dtype=torch.float32, device=dev)
    yv = big[1:].view(ref.shape[0], B)
    yv.copy_(t32(y, dev))
    xg = torch.empty((ref.shape[1], B), dtype=torch.float32, device=dev)
    M.adjoint(yv, xg)
    assert rel(xg.cpu().numpy(), ref.T @ y) <= SPMV_TOL
