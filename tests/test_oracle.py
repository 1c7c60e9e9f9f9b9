"""Pins for the FP64 oracle (CPU only).

Each test checks the oracle against something other than itself: closed forms
derived by hand (tests/golden/closed_forms.json), independent library routines
(scipy's quaternion rotation and Gaussian density, finite-difference
Jacobians), brute force over every label assignment of the paper's integer
program, and invariants of alpha compositing.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle.assign import assign, assign_margin, labels_from_membership
from paper_2409_08270_gb300 import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def _cam(width=32, height=32, fx=40.0, fy=None, cx=None, cy=None, R=None, t=None):
    return {"R": np.eye(3) if R is None else R, "t": np.zeros(3) if t is None else t,
            "fx": fx, "fy": fx if fy is None else fy,
            "cx": width / 2 if cx is None else cx, "cy": height / 2 if cy is None else cy,
            "width": width, "height": height}


def _gauss(means, quats=None, scales=None, opac=None):
    means = np.asarray(means, np.float32).reshape(-1, 3)
    n = means.shape[0]
    quats = np.tile([1, 0, 0, 0], (n, 1)) if quats is None else quats
    scales = np.full((n, 3), 0.1) if scales is None else scales
    opac = np.full(n, 0.5) if opac is None else opac
    return {"mean": means, "quat": np.asarray(quats, np.float32).reshape(-1, 4),
            "scale": np.asarray(scales, np.float32).reshape(-1, 3),
            "opacity": np.asarray(opac, np.float32).reshape(-1)}


def _conic_to_cov(row):
    a, b, c = row[4], row[5], row[6]
    C = np.array([[a, b], [b, c]])
    return np.linalg.inv(C)


# --------------------------------------------------------------------------
# projection (Sec. 3.1: 3D Gaussians projected to 2D Gaussians)
# --------------------------------------------------------------------------

def test_projection_isotropic_on_axis():
    """Isotropic Gaussian on the optical axis: Sigma2D = diag((fx s/z)^2, (fy s/z)^2) + 0.3."""
    z, s = 2.5, 0.07
    cam = _cam(64, 48, fx=55.0, fy=71.0, cx=30.0, cy=20.0)
    g = _gauss([[0, 0, z]], quats=[[0.3, -0.5, 0.2, 0.7]], scales=[[s, s, s]], opac=[0.8])
    row = oracle.project_view(g, cam)[0]
    assert row[0] == 1
    z32, s32 = float(np.float32(z)), float(np.float32(s))
    assert row[1] == pytest.approx(z32, rel=1e-15)
    assert row[2] == pytest.approx(30.0, abs=1e-12) and row[3] == pytest.approx(20.0, abs=1e-12)
    cov = _conic_to_cov(row)
    exp = np.diag([(55.0 * s32 / z32) ** 2 + 0.3, (71.0 * s32 / z32) ** 2 + 0.3])
    np.testing.assert_allclose(cov, exp, rtol=1e-12, atol=1e-14)


def _rot_scipy(q_wxyz):
    from scipy.spatial.transform import Rotation
    w, x, y, z = q_wxyz
    return Rotation.from_quat([x, y, z, w]).as_matrix()      # scipy is scalar-last


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_projection_matches_finite_difference_jacobian(seed):
    """Sigma2D = J W Sigma3D W^T J^T + 0.3 I with J the Jacobian of the pinhole
    map, here taken by central differences, and Sigma3D built with scipy's
    quaternion->matrix (scalar-last convention, converted)."""
    rng = np.random.default_rng(seed)
    cam = synth.camera(rng.uniform(-1, 1, 3) + np.array([0, 0, -4.0]), 200, 150, 180.0,
                       target=rng.uniform(-0.2, 0.2, 3))
    m = rng.uniform(-0.5, 0.5, 3)
    q = rng.standard_normal(4)
    s = np.exp(rng.normal(-2.5, 0.6, 3))
    g = _gauss([m], quats=[q], scales=[s], opac=[0.9])
    row = oracle.project_view(g, cam)[0]
    assert row[0] == 1
    m64, q64, s64 = (np.asarray(g[k][0], np.float64) for k in ("mean", "quat", "scale"))
    R, t = np.asarray(cam["R"]), np.asarray(cam["t"])
    X = R @ m64 + t

    def pin(P):
        return np.array([cam["fx"] * P[0] / P[2] + cam["cx"], cam["fy"] * P[1] / P[2] + cam["cy"]])

    h = 1e-6
    J = np.stack([(pin(X + h * e) - pin(X - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
    Rq = _rot_scipy(q64 / np.linalg.norm(q64))
    S3 = Rq @ np.diag(s64 ** 2) @ Rq.T
    S2 = J @ R @ S3 @ R.T @ J.T + 0.3 * np.eye(2)
    np.testing.assert_allclose(_conic_to_cov(row), S2, rtol=2e-7)
    np.testing.assert_allclose(row[2:4], pin(X), rtol=1e-12)
    assert row[1] == pytest.approx(X[2], rel=1e-14)


def test_identity_and_quarter_turn_quaternion():
    """q = identity keeps the scale axes; a quarter turn about z swaps x and y."""
    z = 3.0
    cam = _cam(64, 64, fx=50.0, fy=50.0)
    a, b, c = 0.05, 0.12, 0.2
    h = math.sqrt(0.5)
    g = _gauss([[0, 0, z], [0, 0, z]], quats=[[1, 0, 0, 0], [h, 0, 0, h]],
               scales=[[a, b, c], [a, b, c]], opac=[0.5, 0.5])
    rows = oracle.project_view(g, cam)
    a32, b32 = float(np.float32(a)), float(np.float32(b))
    exp0 = np.diag([(50 * a32 / z) ** 2 + 0.3, (50 * b32 / z) ** 2 + 0.3])
    exp1 = np.diag([(50 * b32 / z) ** 2 + 0.3, (50 * a32 / z) ** 2 + 0.3])
    np.testing.assert_allclose(_conic_to_cov(rows[0]), exp0, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(_conic_to_cov(rows[1]), exp1, rtol=1e-6, atol=1e-9)


def test_projection_culls():
    cam = _cam()
    g = _gauss([[0, 0, 0.1], [0, 0, 2.0], [0, 0, 2.0], [50, 0, 2.0]],
               opac=[0.5, 0.5, 1.0 / 256.0, 0.5])
    rows = oracle.project_view(g, cam)
    assert rows[:, 0].tolist() == [0, 1, 0, 0]   # near plane, kept, opacity < 1/255, off-screen
    with pytest.raises(ValueError):
        oracle.project_view(_gauss([[0, 0, 2]], quats=[[0, 0, 0, 0]]), cam)


# --------------------------------------------------------------------------
# alpha compositing (Sec. 3.1 Eq. 1)
# --------------------------------------------------------------------------

def test_single_gaussian_alpha_is_unnormalised_density():
    """alpha = min(0.99, o * 2 pi sqrt(det Sigma) * N(d; 0, Sigma)) with scipy's density;
    pixels below 1/255 contribute nothing."""
    from scipy.stats import multivariate_normal
    cam = _cam(40, 36, fx=60.0, fy=48.0, cx=19.5, cy=17.5)   # mean on pixel (19, 17)'s centre
    g = _gauss([[0.0, 0.0, 2.0]], quats=[[0.9, 0.1, -0.3, 0.2]], scales=[[0.12, 0.03, 0.07]],
               opac=[0.995])
    row = oracle.project_view(g, cam)[0]
    cov = _conic_to_cov(row)
    offs, gidx, con, tf = oracle.pixel_lists(g, [cam])
    H, W = 36, 40
    yy, xx = np.mgrid[0:H, 0:W]
    pts = np.stack([xx.ravel() + 0.5, yy.ravel() + 0.5], axis=1)
    dens = multivariate_normal(mean=row[2:4], cov=cov).pdf(pts) * 2 * np.pi * np.sqrt(np.linalg.det(cov))
    alpha = np.minimum(0.99, float(np.float32(0.995)) * dens)
    exp = np.where(alpha >= 1 / 255, alpha, 0.0)
    got = np.zeros(H * W)
    counts = np.diff(offs)
    assert counts.max() <= 1
    got[counts == 1] = con
    np.testing.assert_allclose(got, exp, rtol=1e-12, atol=0)
    assert (got > 0).sum() > 50 and (got == 0.99).sum() > 0   # both the clamp and the cut occur
    np.testing.assert_allclose(tf, 1 - got, rtol=0, atol=1e-15)


def test_opaque_stack_golden():
    gd = GOLDEN["opaque_stack"]
    cam = _cam(17, 17, fx=40.0, cx=8.5, cy=8.5)       # the mean lands on pixel (8, 8)'s centre
    g = _gauss([[0, 0, 2.0]] * gd["count"], scales=np.full((3, 3), 0.05),
               opac=[gd["opacity"]] * gd["count"])
    offs, gidx, con, tf = oracle.pixel_lists(g, [cam])
    p = 8 * 17 + 8
    assert con[offs[p]:offs[p + 1]].tolist() == gd["contributions"]
    assert gidx[offs[p]:offs[p + 1]].tolist() == [0, 1]      # equal depth: lower index first
    assert tf[p] == gd["t_final"]


def test_two_layer_golden_and_depth_order():
    gd = GOLDEN["two_layer"]
    cam = _cam(17, 17, fx=40.0, cx=8.5, cy=8.5)
    # index 0 is the BACK Gaussian: depth, not index, decides the order
    g = _gauss([[0, 0, 3.0], [0, 0, 2.0]], scales=np.full((2, 3), 0.05),
               opac=[gd["opacity_back"], gd["opacity_front"]])
    offs, gidx, con, tf = oracle.pixel_lists(g, [cam])
    p = 8 * 17 + 8
    assert gidx[offs[p]:offs[p + 1]].tolist() == [1, 0]
    assert con[offs[p]:offs[p + 1]].tolist() == gd["contributions"]
    assert tf[p] == gd["t_final"]


def test_compositing_invariant_and_table_consistency(tiny):
    """sum_i alpha_i T_i + T_final = 1 at every pixel; the table equals the
    per-pixel terms binned by label; table total = sum_p (1 - T_final)."""
    cams, masks = tiny.cams[:3], tiny.masks[:3]
    offs, gidx, con, tf = oracle.pixel_lists(tiny.gaussians, cams)
    per_pix = np.add.reduceat(np.append(con, 0.0), offs[:-1]) * (np.diff(offs) > 0)
    np.testing.assert_allclose(per_pix + tf, 1.0, rtol=0, atol=1e-12)
    acc = oracle.accumulate(tiny.gaussians, cams, masks, tiny.E, want_t_final=True)
    np.testing.assert_array_equal(acc.t_final, tf)
    labels = np.concatenate([m.reshape(-1) for m in masks]).astype(np.int64)
    pix_of = np.repeat(np.arange(labels.size), np.diff(offs))
    exp = np.zeros((tiny.n, tiny.E))
    np.add.at(exp, (gidx, labels[pix_of]), con)
    np.testing.assert_allclose(acc.table, exp, rtol=1e-12, atol=1e-15)
    assert acc.table.sum() == pytest.approx((1 - tf).sum(), rel=1e-12)


def test_spatial_index_equals_brute_force(tiny):
    """cull_mode=1 walks every projected Gaussian at every pixel (no spatial
    index); the table, flags and transmittance must be identical."""
    a = oracle.accumulate(tiny.gaussians, tiny.cams[:4], tiny.masks[:4], tiny.E, want_t_final=True)
    b = oracle.accumulate(tiny.gaussians, tiny.cams[:4], tiny.masks[:4], tiny.E, cull_mode=1,
                          want_t_final=True)
    np.testing.assert_array_equal(a.table, b.table)
    np.testing.assert_array_equal(a.t_final, b.t_final)
    assert b.n_eval > 5 * a.n_eval


def test_brute_force_clustered_scene():
    w = synth.binary_scene(n=3000, views=2, width=96, height=72, n_clusters=4)
    a = oracle.accumulate(w.gaussians, w.cams, w.masks, w.E)
    b = oracle.accumulate(w.gaussians, w.cams, w.masks, w.E, cull_mode=1)
    np.testing.assert_array_equal(a.table, b.table)


def test_thread_count_and_selection(tiny):
    a = oracle.accumulate(tiny.gaussians, tiny.cams, tiny.masks, tiny.E, nthreads=1)
    b = oracle.accumulate(tiny.gaussians, tiny.cams, tiny.masks, tiny.E, nthreads=5)
    np.testing.assert_allclose(a.table, b.table, rtol=1e-13, atol=1e-16)
    sel = np.array([3, 17, 400, 1999])
    c = oracle.accumulate(tiny.gaussians, tiny.cams, tiny.masks, tiny.E, sel=sel)
    np.testing.assert_allclose(c.table, a.table[sel], rtol=1e-13, atol=1e-16)


def test_tracked_rows_equal_full_walk_on_clustered_scene():
    """Tracked rows (each Gaussian walked over its own box, candidates from a
    coarse grid of the view) equal the full walk's rows on a clustered scene
    whose footprints span many grid cells, small and large ones alike."""
    w = synth.binary_scene(n=20000, views=2, width=320, height=240)
    full = oracle.accumulate(w.gaussians, w.cams, w.masks, w.E)
    seen = np.flatnonzero(full.table.sum(1) > 0)
    area = np.zeros(w.n)
    for cam in w.cams:
        pv = oracle.project_view(w.gaussians, cam)
        area = np.maximum(area, pv[:, 8] * pv[:, 9])
    big = seen[np.argsort(-area[seen])[:20]]
    rng = np.random.default_rng(2)
    sel = np.unique(np.concatenate([big, rng.choice(seen, 80, replace=False)]))
    assert area[big].min() > 64 * 64
    t = oracle.accumulate(w.gaussians, w.cams, w.masks, w.E, sel=sel)
    np.testing.assert_allclose(t.table, full.table[sel], rtol=1e-12, atol=1e-15)


def test_column_sums_independent_of_labels(tiny):
    """sum_e A[i, e] depends on the scene and cameras only; relabelling the
    masks permutes the columns."""
    E = 3
    rng = np.random.default_rng(5)
    m1 = [rng.integers(0, E, size=m.shape) for m in tiny.masks]
    m2 = [np.zeros_like(m) for m in tiny.masks]
    perm = np.array([2, 0, 1])
    m3 = [perm[m] for m in m1]
    a1 = oracle.accumulate(tiny.gaussians, tiny.cams, m1, E).table
    a2 = oracle.accumulate(tiny.gaussians, tiny.cams, m2, E).table
    a3 = oracle.accumulate(tiny.gaussians, tiny.cams, m3, E).table
    np.testing.assert_allclose(a1.sum(1), a2.sum(1), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(a3[:, perm], a1, rtol=1e-12, atol=1e-15)


def test_bad_labels_are_skipped(tiny):
    masks = [m.astype(np.int32) for m in tiny.masks[:2]]
    masks[0] = masks[0].copy()
    masks[0][:4, :] = 7
    masks[1] = masks[1].copy()
    masks[1][:, :2] = -1
    acc = oracle.accumulate(tiny.gaussians, tiny.cams[:2], masks, 2)
    assert acc.n_bad_label == 4 * 128 + 2 * 128
    ref = oracle.accumulate(tiny.gaussians, tiny.cams[:2], [m.clip(0, 1) for m in masks], 2)
    assert acc.table.sum() < ref.table.sum()


# --------------------------------------------------------------------------
# the integer program (Sec. 3.2 Eq. 2-6) and its closed form
# --------------------------------------------------------------------------

def _small_scene(seed, n, views, size, E):
    rng = np.random.default_rng(seed)
    g = {
        "mean": rng.uniform(-0.35, 0.35, (n, 3)).astype(np.float32),
        "quat": rng.standard_normal((n, 4)).astype(np.float32),
        "scale": np.exp(rng.normal(-2.0, 0.4, (n, 3))).astype(np.float32),
        "opacity": rng.uniform(0.2, 0.99, n).astype(np.float32),
    }
    cams = []
    for v in range(views):
        az = 2 * math.pi * v / views + 0.3
        cams.append(synth.camera((2.0 * math.sin(az), 0.4, -2.0 * math.cos(az)), size, size,
                                 size * 1.1))
    masks = [rng.integers(0, E, size=(size, size)) for _ in range(views)]
    # blobs make the vote non-trivial: most pixels agree locally
    for m in masks:
        yy, xx = np.mgrid[0:size, 0:size]
        m[(xx - size / 2) ** 2 + (yy - size / 2.5) ** 2 < (size / 4) ** 2] = E - 1
    return g, cams, masks


def _dense_terms(g, cams):
    offs, gidx, con, tf = oracle.pixel_lists(g, cams)
    n = g["mean"].shape[0]
    P = offs.size - 1
    C = np.zeros((n, P))
    pix = np.repeat(np.arange(P), np.diff(offs))
    np.add.at(C, (gidx, pix), con)
    return C


@pytest.mark.parametrize("seed,n,views,size,E", [
    (11, 10, 2, 24, 2), (12, 12, 3, 16, 2), (13, 9, 4, 20, 3), (14, 12, 1, 48, 3), (15, 11, 2, 32, 2),
])
def test_closed_form_reaches_ilp_optimum(seed, n, views, size, E):
    """Brute force over all 2^N assignments.  For label e, with y_p = [M_p = e]
    and x_p = sum_i P_i alpha_i T_i rendered per pixel (Eq. 1 with x_i = P_i),
    the objective of Eq. 2 (gamma = 0) and its background-biased form
    F_gamma = sum_p w_p |x_p - y_p|, w_p = (1 - gamma) if y_p else (1 + gamma),
    is minimised by the closed-form membership S[e] (Eq. 6/7 with the bias)."""
    g, cams, masks = _small_scene(seed, n, views, size, E)
    C = _dense_terms(g, cams)                                 # [N, P]
    lab = np.concatenate([m.reshape(-1) for m in masks])
    A = oracle.accumulate(g, cams, masks, E).table
    Pall = np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.float64)   # [2^N, N]
    X = Pall @ C                                               # rendered masks, [2^N, P]
    assert X.max() <= 1 + 1e-12 and X.min() >= 0                # Lemma 1
    for gamma in GOLDEN["gamma_grid"]["values"]:
        S = assign(A, gamma)
        for e in range(E):
            y = (lab == e).astype(np.float64)
            wts = np.where(y > 0, 1 - gamma, 1 + gamma)
            F = (np.abs(X - y[None, :]) * wts[None, :]).sum(1)
            k = int(np.dot(S[e].astype(np.int64), 1 << np.arange(n - 1, -1, -1)))
            assert F[k] <= F.min() * (1 + 1e-12) + 1e-12, (gamma, e, F[k], F.min())
            # unique minimiser when every coefficient is clearly non-zero
            coef = (1 + gamma) * (A.sum(1) - A[:, e]) - (1 - gamma) * A[:, e]
            if np.all(np.abs(coef) > 1e-9):
                assert int(np.argmin(F)) == k


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_linearisation_eq3_to_eq5(seed):
    """F(P) evaluated per pixel equals C + sum_i P_i (A_0^i - A_1^i) (Eq. 3-5),
    and the rendered total equals sum_i P_i sum_e A[i, e]."""
    g, cams, masks = _small_scene(seed, 12, 3, 24, 2)
    C = _dense_terms(g, cams)
    lab = np.concatenate([m.reshape(-1) for m in masks]).astype(np.float64)
    A = oracle.accumulate(g, cams, masks, 2).table
    rng = np.random.default_rng(seed)
    for _ in range(20):
        P = rng.integers(0, 2, 12).astype(np.float64)
        x = P @ C
        F = np.abs(x - lab).sum()
        np.testing.assert_allclose(F, lab.sum() + P @ (A[:, 0] - A[:, 1]), rtol=1e-12)
        np.testing.assert_allclose(x.sum(), P @ A.sum(1), rtol=1e-12)


# --------------------------------------------------------------------------
# the assignment (Sec. 3.2 regularised ILP, Sec. 3.3 Eq. 7, Listing 1)
# --------------------------------------------------------------------------

def test_assign_golden_ties():
    for case in GOLDEN["assign_ties"]["cases"]:
        S = assign(np.array([case["A"]]), case["gamma"])
        assert bool(S[1, 0]) == case["member_label1"], case


@pytest.mark.parametrize("gamma", GOLDEN["gamma_grid"]["values"] + GOLDEN["gamma_grid"]["ends"])
def test_assign_threshold_law(gamma):
    """Membership of e  <=>  A_e > (1 + gamma)/2 * sum_e A  (sum > 0), and
    <=> gamma < 0 for a Gaussian nobody saw; exclusive for gamma >= 0."""
    rng = np.random.default_rng(7)
    A = rng.exponential(1.0, (5000, 6)) * (rng.random((5000, 6)) < 0.6)
    A[:50] = 0.0
    S = assign(A, gamma)
    s = A.sum(1)
    for e in range(6):
        exp = np.where(s > 0, A[:, e] > (1 + gamma) / 2 * s, gamma < 0)
        # only exact ties could differ in rounding; the random table has none
        np.testing.assert_array_equal(S[e], exp)
    if gamma >= 0:
        assert S.sum(0).max() <= 1
    if gamma == 1.0:
        assert not S.any()
    if gamma == -1.0:
        np.testing.assert_array_equal(S, (A > 0).T | (s == 0)[None, :])


def _normalise_bias_argmax(A, gamma):
    """The multi-instance assignment as Supp. Sec. 6 states its steps, with
    torch's own primitives in float64: the row sum is taken once; for every
    object the pair (others, object) is L1-normalised over the pair (torch's
    F.normalize, p = 1, default epsilon), the bias is added to the "others"
    entry and the argmax (first maximum) decides membership."""
    import torch
    import torch.nn.functional as F
    t = torch.from_numpy(np.asarray(A, dtype=np.float64)).T      # [E, N]
    total = t.sum(0)
    rows = []
    for e in range(t.shape[0]):
        pair = torch.stack([total - t[e], t[e]])                 # [2, N]
        pair = F.normalize(pair, p=1, dim=0)
        pair[0] += gamma
        rows.append(torch.argmax(pair, dim=0) == 1)
    return torch.stack(rows).numpy()


@pytest.mark.parametrize("gamma", GOLDEN["gamma_grid"]["values"] + GOLDEN["gamma_grid"]["ends"])
def test_assign_equals_normalise_bias_argmax(gamma, tiny):
    """The oracle's closed-form rule gives the same segmentation matrix as
    the normalise / bias / argmax procedure run with torch, on oracle tables
    (binary and multi-label, unseen rows included) and on a random table with
    rows far below the normalisation epsilon."""
    acc2 = oracle.accumulate(tiny.gaussians, tiny.cams[:3], tiny.masks[:3], 2)
    rng = np.random.default_rng(4)
    masks4 = [rng.integers(0, 4, m.shape).astype(np.int32) for m in tiny.masks[:3]]
    acc4 = oracle.accumulate(tiny.gaussians, tiny.cams[:3], masks4, 4)
    R = rng.exponential(1.0, (3000, 5)) * (rng.random((3000, 5)) < 0.5)
    R[:300] *= 1e-15                                              # below epsilon = 1e-12
    R[300:320] = 0.0
    for A in (acc2.table, acc4.table, R):
        A = np.vstack([A, np.zeros((3, A.shape[1]))])             # three unseen Gaussians
        np.testing.assert_array_equal(assign(A, gamma), _normalise_bias_argmax(A, gamma))


def test_assign_overlap_only_below_zero():
    A = np.array([[1.0, 1.0, 1.0], [2.0, 1.0, 1.0]])
    assert assign(A, -0.5)[:, 0].sum() == 3       # Sec. 3.3: subsets overlap for gamma < 0
    assert assign(A, 0.0)[:, 0].sum() == 0
    assert assign(A, 0.0)[:, 1].tolist() == [False, False, False]
    assert assign(A, -0.2)[:, 1].tolist() == [True, False, False]


def test_assign_margin_and_labels():
    A = np.array([[1.0, 3.0], [3.0, 1.0], [0.0, 0.0], [1.0, 1.0]])
    m = assign_margin(A, 0.5)
    # (1-g)A_e - (1+g)(S-A_e) over S: label 1 of row 0: (0.5*3 - 1.5*1)/4 = 0
    assert m[0, 1] == 0.0 and m[0, 0] == pytest.approx((1.5 * 3 - 0.5 * 1) / 4)
    assert np.isinf(m[2]).all()
    lab = labels_from_membership(assign(A, 0.0))
    assert lab.tolist() == [1, 0, -1, -1]


def test_special_masks(tiny):
    """All-foreground masks: every seen Gaussian joins label 1 (gamma < 1);
    all-background: none does."""
    cams = tiny.cams[:3]
    fg = oracle.accumulate(tiny.gaussians, cams, [np.ones_like(m) for m in tiny.masks[:3]], 2)
    bg = oracle.accumulate(tiny.gaussians, cams, [np.zeros_like(m) for m in tiny.masks[:3]], 2)
    seen = fg.table.sum(1) > 0
    assert seen.sum() > 100
    for gamma in (-0.8, 0.0, 0.9):
        assert assign(fg.table, gamma)[1][seen].all()
        assert not assign(bg.table, gamma)[1][seen].any()


def _on_axis_scene(means_z, opac, sigma_px, width=24, fx=20.0):
    """Isotropic Gaussians on the optical axis of a camera at the origin
    looking down +z, with projected standard deviation sigma_px pixels."""
    n = len(means_z)
    z = np.asarray(means_z, np.float64)
    s = np.asarray(sigma_px, np.float64) * z / fx
    g = {"mean": np.column_stack([np.zeros(n), np.zeros(n), z]).astype(np.float32),
         "quat": np.tile([1, 0, 0, 0], (n, 1)).astype(np.float32),
         "scale": np.repeat(s[:, None], 3, axis=1).astype(np.float32),
         "opacity": np.asarray(opac, np.float32)}
    cam = {"R": np.eye(3), "t": np.zeros(3), "fx": fx, "fy": fx, "cx": width / 2,
           "cy": width / 2, "width": width, "height": width}
    return g, [cam]


def _risk_scenes(tiny):
    """Scenes where many decisions sit on their thresholds."""
    scenes = {}
    # four layers of opacity o over the whole view: T after the fourth factor
    # is 1e-4 (1 - 2.5e-5) at the centre and rises by ~5e-5 relative towards
    # the corners, so the stop decision of the fourth layer is marginal
    Tc = 1e-4 * (1 - 2.5e-5)
    o = 1 - Tc ** 0.25
    scenes["stop_stack"] = _on_axis_scene([2.0, 2.5, 3.0, 3.5], [o] * 4, [1.0e4] * 4)
    # one Gaussian whose alpha straddles 1/255 within 3e-5 across the view,
    # and an opaque-ish layer behind it
    scenes["alpha_ring"] = _on_axis_scene([2.0, 3.0], [(1 + 3e-5) / 255, 0.5], [1.55e3, 30.0])
    # two Gaussians at exactly the same depth
    scenes["tie"] = _on_axis_scene([2.0, 2.0, 3.0], [0.6, 0.7, 0.5], [6.0, 9.0, 20.0])
    scenes["tiny"] = (tiny.gaussians, tiny.cams[:2])
    return scenes


def test_risk_bounds_the_change_when_decisions_flip(tiny):
    """The per-entry risk is a bound: moving the 1/255 and 1e-4 thresholds by
    0.9 of the alpha window (up and down), or walking equal depths in the
    other order, changes no table entry by more than its risk.  Each kind of
    move does change some entry, so the bound is exercised."""
    eps = 1e-5
    moves = {"alpha_up": {"alpha_min": (1 + 0.9 * eps) / 255},
             "alpha_down": {"alpha_min": (1 - 0.9 * eps) / 255},
             "t_up": {"t_min": 1e-4 * (1 + 0.9 * eps)},
             "t_down": {"t_min": 1e-4 * (1 - 0.9 * eps)},
             "ties": {"tie_reverse": True}}
    changed = {k: 0 for k in moves}
    for name, (g, cams) in _risk_scenes(tiny).items():
        rng = np.random.default_rng(8)
        masks = [rng.integers(0, 3, (c["height"], c["width"])).astype(np.int32) for c in cams]
        base = oracle.accumulate(g, cams, masks, 3, event_rel=eps)
        scale = np.abs(base.table).max()
        for k, kw in moves.items():
            alt = oracle.accumulate(g, cams, masks, 3, event_rel=eps, **kw)
            diff = np.abs(alt.table - base.table)
            bad = diff > base.risk * (1 + 1e-9) + 1e-14 * scale
            assert not bad.any(), (name, k, np.argwhere(bad)[:5], diff[bad][:5], base.risk[bad][:5])
            changed[k] += int((diff > 1e-12 * scale).sum())
    print("entries moved per kind of decision change:", changed)
    assert all(v > 0 for v in changed.values()), changed


def test_risk_window_narrower_than_the_move_fails(tiny):
    """The check above can fail: with windows narrower than the threshold
    move, flipped decisions are no longer marked marginal and the change
    exceeds the risk.  (The window of the stop decision is the alpha
    precision amplified by the factors of T, about 37-fold in the stack.)"""
    for name, er in (("alpha_ring", 1e-6), ("stop_stack", 1e-8)):
        g, cams = _risk_scenes(tiny)[name]
        masks = [np.ones((c["height"], c["width"]), np.int32) for c in cams]
        base = oracle.accumulate(g, cams, masks, 2, event_rel=er)
        kw = {"alpha_min": (1 - 9e-6) / 255} if name == "alpha_ring" else {"t_min": 1e-4 * (1 + 9e-6)}
        alt = oracle.accumulate(g, cams, masks, 2, event_rel=er, **kw)
        assert (np.abs(alt.table - base.table) > base.risk * (1 + 1e-9)).any(), name


def test_risk_bounds_are_local(tiny):
    """The near-threshold bookkeeping stays small relative to the
    contributions, so the parity comparison stays tight for almost every
    Gaussian."""
    acc = oracle.accumulate(tiny.gaussians, tiny.cams, tiny.masks, tiny.E)
    s = acc.table.sum(1)
    r = acc.risk.sum(1)
    rel = r[s > 0] / s[s > 0]
    assert np.median(rel) < 1e-5
    assert (rel > 1e-3).mean() < 0.01


def test_event_window_changes_risk_only(tiny):
    """The near-threshold window shapes the risk bookkeeping, never the table:
    a narrower window gives the same FP64 table and no more risk."""
    a = oracle.accumulate(tiny.gaussians, tiny.cams[:3], tiny.masks[:3], tiny.E)
    b = oracle.accumulate(tiny.gaussians, tiny.cams[:3], tiny.masks[:3], tiny.E, event_rel=1e-9)
    assert np.array_equal(a.table, b.table)
    assert b.risk.sum() <= a.risk.sum()
    assert (b.risk > 0).sum() < (a.risk > 0).sum()


# --------------------------------------------------------------------------
# reduced-precision record (FP16 whitening matrix, FP32 mean)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("theta,sx,sy,o", [(0.0, 0.05, 0.05, 0.7), (0.6, 0.08, 0.02, 0.9),
                                           (-1.1, 0.03, 0.11, 0.995)])
def test_record_f16_closed_form(theta, sx, sy, o):
    """One Gaussian on the optical axis, rotated by theta about z: Sigma2D =
    (f/z)^2 R(theta) diag(sx^2, sy^2) R(theta)^T + 0.3 I exactly.  Its
    whitening matrix is formed here from that closed form (major unit
    eigenvector (h + r, b) / |.| for h >= 0, else (b, r - h) / |.|), rounded
    with numpy's float16, and sum_p min(0.99, o 2^-|W (p - m)|^2) over the
    pixels where alpha >= 1/255 must equal the table (T = 1 throughout)."""
    z, f, W_, H_ = 2.0, 60.0, 48, 40
    q = [math.cos(theta / 2), 0.0, 0.0, math.sin(theta / 2)]
    g = _gauss([[0.0, 0.0, z]], quats=[q], scales=[[sx, sy, 0.05]], opac=[o])
    cam = _cam(W_, H_, fx=f, cx=W_ / 2 + 0.3, cy=H_ / 2 - 0.2)
    acc = oracle.accumulate(g, [cam], [np.ones((H_, W_), np.int32)], 2, record_f16=True)
    s32 = np.float32([sx, sy])
    R2 = np.array([[math.cos(theta), -math.sin(theta)], [math.sin(theta), math.cos(theta)]])
    S = (f / z) ** 2 * R2 @ np.diag(np.float64(s32) ** 2) @ R2.T + 0.3 * np.eye(2)
    a, b, c = S[0, 0], S[0, 1], S[1, 1]
    h = 0.5 * (a - c)
    r = math.hypot(h, b)
    l1 = 0.5 * (a + c) + r
    l2 = (a * c - b * b) / l1
    e = np.array([h + r, b]) if h >= 0 else np.array([b, r - h])
    e = e / np.linalg.norm(e) if np.linalg.norm(e) > 0 else np.array([1.0, 0.0])
    k = np.sqrt(0.5 * math.log2(math.e) / np.array([l1, l2]))
    W = np.array([[e[0] * k[0], e[1] * k[0]], [-e[1] * k[1], e[0] * k[1]]])
    W16 = W.astype(np.float16).astype(np.float64)
    m = np.array([np.float32(cam["cx"]), np.float32(cam["cy"])], np.float64)
    ys, xs = np.mgrid[0:H_, 0:W_]
    d = np.stack([xs + 0.5 - m[0], ys + 0.5 - m[1]], -1)
    w = d @ W16.T
    alpha = np.minimum(0.99, np.float64(np.float32(o)) * np.exp2(-(w ** 2).sum(-1)))
    expect = alpha[alpha >= 1 / 255].sum()
    assert acc.table[0, 1] == pytest.approx(expect, rel=1e-12)
    # rounding W to FP16 moves the sum, but by far less than the 1/255 cut
    plain = oracle.accumulate(g, [cam], [np.ones((H_, W_), np.int32)], 2)
    assert acc.table[0, 1] == pytest.approx(plain.table[0, 1], rel=2e-2)


def test_record_f16_close_to_plain(tiny):
    """The FP16 record perturbs alpha by ~1e-3 relative: the tables agree to
    a few per cent on every substantial entry and the labels on nearly all."""
    a = oracle.accumulate(tiny.gaussians, tiny.cams[:3], tiny.masks[:3], tiny.E)
    b = oracle.accumulate(tiny.gaussians, tiny.cams[:3], tiny.masks[:3], tiny.E, record_f16=True)
    big = a.table > 1e-3 * a.table.max()
    rel = np.abs(b.table[big] - a.table[big]) / a.table[big]
    assert np.median(rel) < 5e-3 and rel.max() < 0.2
    assert not np.array_equal(a.table, b.table)
    agree = (assign(a.table, tiny.gamma) == assign(b.table, tiny.gamma)).mean()
    assert agree > 0.99


# --------------------------------------------------------------------------
# 3-sigma tile coverage (the standard rasteriser's, reused by the paper, Sec. 4.2)
# --------------------------------------------------------------------------

def _brute_render_3sigma(g, cam, mask, E):
    """Every pixel against every Gaussian in (depth, index) order, Eq. 1 with
    the skip and stop rules; a Gaussian is seen only in the 16x16 tiles that
    the square of half side ceil(3 sqrt(lambda_max(Sigma2D))) around its
    projected mean overlaps."""
    pv = oracle.project_view(g, cam)
    N = pv.shape[0]
    table = np.zeros((N, E))
    valid = np.flatnonzero(pv[:, 0] > 0)
    order = valid[np.lexsort((valid, pv[valid, 1]))]
    rect = {}
    for i in order:
        a, b, c = pv[i, 4], pv[i, 5], pv[i, 6]
        S = np.linalg.inv(np.array([[a, b], [b, c]]))
        r = np.ceil(3 * np.sqrt(np.linalg.eigvalsh(S).max()))
        mx, my = pv[i, 2], pv[i, 3]
        rect[i] = (np.floor((mx - r) / 16), np.ceil((mx + r) / 16) - 1,
                   np.floor((my - r) / 16), np.ceil((my + r) / 16) - 1)
    for v in range(cam["height"]):
        for u in range(cam["width"]):
            T = 1.0
            for i in order:
                tx0, tx1, ty0, ty1 = rect[i]
                if not (tx0 <= u // 16 <= tx1 and ty0 <= v // 16 <= ty1):
                    continue
                dx, dy = u + 0.5 - pv[i, 2], v + 0.5 - pv[i, 3]
                power = -0.5 * (pv[i, 4] * dx * dx + pv[i, 6] * dy * dy) - pv[i, 5] * dx * dy
                alpha = min(0.99, pv[i, 7] * np.exp(power))
                if alpha < 1 / 255:
                    continue
                if T * (1 - alpha) < 1e-4:
                    break
                table[i, mask[v, u]] += alpha * T
                T *= 1 - alpha
    return table


def test_3sigma_coverage_matches_brute_force():
    """Opaque Gaussians elongated along the image x axis (their alpha >= 1/255
    ellipse reaches 3.3 sigma there, past the 3-sigma square) on a 64x48 view:
    the oracle's 3-sigma mode equals the brute-force renderer, and it differs
    from the exact coverage on several Gaussians."""
    rng = np.random.default_rng(5)
    n = 16
    quat = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1))
    quat[:, 3] = rng.uniform(-0.05, 0.05, n)
    g = {"mean": np.column_stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.5, 0.5, n),
                                  rng.uniform(-0.3, 0.3, n)]).astype(np.float32),
         "quat": quat,
         "scale": np.column_stack([rng.uniform(0.15, 0.3, n), rng.uniform(0.02, 0.06, n),
                                   rng.uniform(0.02, 0.06, n)]).astype(np.float32),
         "opacity": rng.uniform(0.95, 0.99, n).astype(np.float32)}
    cam = synth.camera((0.0, 0.0, -3.0), 64, 48, 120.0)
    mask = rng.integers(0, 2, (48, 64)).astype(np.int32)
    ora = oracle.accumulate(g, [cam], [mask], 2, coverage=oracle.COVERAGE_3SIGMA)
    ref = _brute_render_3sigma(g, cam, mask, 2)
    np.testing.assert_allclose(ora.table, ref, rtol=1e-10, atol=1e-14)
    exact = oracle.accumulate(g, [cam], [mask], 2)
    moved = np.abs(exact.table - ora.table).sum(1)
    assert (moved > 1e-3).sum() >= 5


def test_3sigma_coverage_equals_exact_for_faint_gaussians(tiny):
    """With every opacity at most 0.3 the alpha >= 1/255 ellipse,
    d^T Sigma^-1 d <= 2 ln(255 o) <= 8.7, lies inside the 3-sigma square, so
    both coverages give the same table."""
    g = dict(tiny.gaussians)
    g["opacity"] = np.minimum(g["opacity"], 0.3).astype(np.float32)
    a = oracle.accumulate(g, tiny.cams[:3], tiny.masks[:3], 2)
    b = oracle.accumulate(g, tiny.cams[:3], tiny.masks[:3], 2, coverage=oracle.COVERAGE_3SIGMA)
    np.testing.assert_array_equal(a.table, b.table)
    assert a.table.sum() > 0


# --------------------------------------------------------------------------
# Novel-view mask rendering (Sec. 3.4; Supp. Sec. 8.2; tau = 0.1, Sec. 4.6)
# --------------------------------------------------------------------------

def _alpha_on_axis(o, sigma_px, width, x, y, z=None, fx=20.0):
    """Closed form: isotropic Gaussian on the axis, Sigma2D = (s^2 + 0.3) I,
    mean at the view centre, pixel (x, y) sampled at its centre.  The scene
    stores FP32 values: o and the scale fx^-1 sigma z are taken as rounded."""
    o = float(np.float32(o))
    if z is not None:
        z32 = float(np.float32(z))
        sigma_px = fx * float(np.float32(sigma_px * z / fx)) / z32
    var = sigma_px ** 2 + 0.3
    dx, dy = x + 0.5 - width / 2, y + 0.5 - width / 2
    a = o * np.exp(-0.5 * (dx * dx + dy * dy) / var)
    return np.where(a >= 1 / 255, np.minimum(a, 0.99), 0.0)


def test_render_one_gaussian_rho_is_alpha_and_binary_mask_is_threshold():
    """One Gaussian in the foreground: rho = alpha at every pixel, D = its
    depth, and the binary mask (E = 2) is [alpha > 0.1]."""
    width, sigma, o, z = 24, 3.0, 0.8, 2.5
    g, cams = _on_axis_scene([z], [o], [sigma], width=width)
    r = oracle.render_masks(g, cams, np.array([0b10], np.uint64), 2, tau=0.1)
    yy, xx = np.mgrid[0:width, 0:width]
    a = _alpha_on_axis(o, sigma, width, xx, yy, z=z)
    np.testing.assert_allclose(r.rho[0][0], a, rtol=1e-12, atol=0)
    assert np.all(r.rho_risk[0][0] == 0)
    np.testing.assert_allclose(r.depth[0][0][a > 0], z, rtol=1e-6)  # the mean's depth (f32 input)
    np.testing.assert_array_equal(r.label[0], (a > 0.1).astype(np.int32))
    assert 0 < (a > 0.1).sum() < (a > 0).sum()
    # not a member: nothing is rendered
    r0 = oracle.render_masks(g, cams, np.array([0b01], np.uint64), 2)
    assert np.all(r0.rho[0] == 0) and np.all(r0.label[0] == 0)


def test_render_each_object_alone_and_front_depth_wins():
    """Two opaque layers in different objects: each object is rendered on its
    own (rho^e = its own alpha, not attenuated by the other layer), both pass
    tau, and the object in front wins; swapping the memberships swaps the
    winner.  A third object behind a transparent layer passes only where its
    own alpha does."""
    width = 16
    g, cams = _on_axis_scene([2.0, 3.0, 4.0], [0.9, 0.95, 0.3], [4.0, 6.0, 3.0], width=width)
    yy, xx = np.mgrid[0:width, 0:width]
    a = [_alpha_on_axis(o, s, width, xx, yy, z=z)
         for o, s, z in ((0.9, 4.0, 2.0), (0.95, 6.0, 3.0), (0.3, 3.0, 4.0))]
    r = oracle.render_masks(g, cams, np.array([1 << 1, 1 << 2, 1 << 3], np.uint64), 4)
    for e in range(3):
        np.testing.assert_allclose(r.rho[0][e], a[e], rtol=1e-12, atol=0)
    want = np.zeros((width, width), np.int32)
    for e, zdep in sorted(((e, d) for e, d in enumerate([2.0, 3.0, 4.0])), key=lambda t: -t[1]):
        want = np.where(a[e] > 0.1, e + 1, want)     # the nearest passing object last
    np.testing.assert_array_equal(r.label[0], want)
    assert {1, 2}.issubset(set(np.unique(r.label[0]).tolist()))
    r2 = oracle.render_masks(g, cams, np.array([1 << 2, 1 << 1, 1 << 3], np.uint64), 4)
    centre = width // 2
    assert r.label[0][centre, centre] == 1 and r2.label[0][centre, centre] == 2


def _brute_subset_render(g, cam, member, e):
    """Per pixel, the Gaussians of object e in (depth, index) order with the
    skip and stop rules: rho = sum alpha T and sum alpha T z."""
    pv = oracle.project_view(g, cam)
    valid = np.flatnonzero((pv[:, 0] > 0) & ((member >> np.uint64(e)) & np.uint64(1) == 1))
    order = valid[np.lexsort((valid, pv[valid, 1]))]
    H, W = cam["height"], cam["width"]
    rho, zs = np.zeros((H, W)), np.zeros((H, W))
    for v in range(H):
        for u in range(W):
            T = 1.0
            for i in order:
                dx, dy = u + 0.5 - pv[i, 2], v + 0.5 - pv[i, 3]
                power = -0.5 * (pv[i, 4] * dx * dx + pv[i, 6] * dy * dy) - pv[i, 5] * dx * dy
                alpha = min(0.99, pv[i, 7] * np.exp(power))
                if alpha < 1 / 255:
                    continue
                if T * (1 - alpha) < 1e-4:
                    break
                rho[v, u] += alpha * T
                zs[v, u] += alpha * T * pv[i, 1]
                T *= 1 - alpha
    return rho, zs


def test_render_matches_brute_force_and_the_rule():
    """A random scene split into three overlapping objects (a Gaussian may
    belong to several): rho^e and sum alpha T z equal a brute-force walk of
    each subset, and every mask value follows the rule -- it passes tau and
    has the smallest depth among the objects that pass, or no object passes."""
    rng = np.random.default_rng(17)
    n = 40
    g = {"mean": np.column_stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.4, 0.4, n),
                                  rng.uniform(-0.5, 0.5, n)]).astype(np.float32),
         "quat": rng.standard_normal((n, 4)).astype(np.float32),
         "scale": rng.uniform(0.03, 0.15, (n, 3)).astype(np.float32),
         "opacity": rng.uniform(0.05, 0.99, n).astype(np.float32)}
    cam = synth.camera((0.3, 0.2, -3.0), 28, 20, 40.0)
    member = np.zeros(n, np.uint64)
    for e in (1, 2, 3):
        member |= (rng.random(n) < 0.45).astype(np.uint64) << np.uint64(e)
    r = oracle.render_masks(g, [cam], member, 4, tau=0.1)
    for e in (1, 2, 3):
        rho, zs = _brute_subset_render(g, cam, member, e)
        np.testing.assert_allclose(r.rho[0][e - 1], rho, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(r.z_sum[0][e - 1], zs, rtol=1e-12, atol=1e-15)
    rho, depth, lab = r.rho[0], r.depth[0], r.label[0]
    passing = rho > 0.1
    for y in range(cam["height"]):
        for x in range(cam["width"]):
            es = [e for e in range(3) if passing[e, y, x]]
            if not es:
                assert lab[y, x] == 0
            else:
                best = min(es, key=lambda e: (depth[e, y, x], e))
                assert lab[y, x] == best + 1
    assert len(np.unique(lab)) == 4               # every object wins somewhere, and 0 too
