"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: Jacobians are checked by
central finite differences of the constraint values (with rotations perturbed
by the exact exponential map), stiffness constants by quadrature of the
paper's disc integrands, and whole steps by closed forms (free fall, twist
decay), invariants (rest state, rigid motions, momentum, unit quaternions),
brute force (pill projection, narrowphase, broadphase) and the paper's
qualitative results (volume held, stretched rods thin).
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1906_05260_gb300 import scenes as S

RNG = np.random.default_rng(1234)


def _rand_quat(rng):
    q = rng.normal(size=4)
    return q / np.linalg.norm(q)


def _rot(q, v):
    return S.quat_rotate(np.asarray(q), np.asarray(v))


def _perturb_rot(q, dth):
    return S.quat_mul(S.axis_angle_quat(np.asarray(dth)), np.asarray(q))


# --------------------------------------------------------------------------
# Jacobians vs central finite differences (Sec. 5, App. A constraints)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4])
def test_segment_jacobians_match_finite_differences(kind):
    rng = np.random.default_rng(10 + kind)
    for _ in range(20):
        xa, xb = rng.normal(size=3), rng.normal(size=3)
        sa, sb = rng.uniform(0.5, 1.5, 2)
        q = _rand_quat(rng)
        lbar = rng.uniform(0.3, 2.0)
        r = oracle.segment_constraint(kind, xa, xb, sa, sb, q, lbar)
        eps = 1e-6
        rows = r["C"].shape[0]

        def C_of(xa_=xa, xb_=xb, sa_=sa, sb_=sb, q_=q):
            return oracle.segment_constraint(kind, xa_, xb_, sa_, sb_, q_, lbar)["C"]

        for c in range(3):
            e = np.zeros(3); e[c] = eps
            fd = (C_of(xa_=xa + e) - C_of(xa_=xa - e)) / (2 * eps)
            np.testing.assert_allclose(r["Jxa"][:, c], fd, rtol=1e-6, atol=1e-7)
            fd = (C_of(xb_=xb + e) - C_of(xb_=xb - e)) / (2 * eps)
            np.testing.assert_allclose(r["Jxb"][:, c], fd, rtol=1e-6, atol=1e-7)
            fd = (C_of(q_=_perturb_rot(q, e)) - C_of(q_=_perturb_rot(q, -e))) / (2 * eps)
            np.testing.assert_allclose(r["Jth"][:, c], fd, rtol=1e-6, atol=1e-7)
        fd = (C_of(sa_=sa + eps) - C_of(sa_=sa - eps)) / (2 * eps)
        np.testing.assert_allclose(r["Jsa"], fd, rtol=1e-6, atol=1e-7)
        fd = (C_of(sb_=sb + eps) - C_of(sb_=sb - eps)) / (2 * eps)
        np.testing.assert_allclose(r["Jsb"], fd, rtol=1e-6, atol=1e-7)
        assert rows == (3 if kind in (0, 4) else 1)


@pytest.mark.parametrize("kind", [0, 1])
def test_vertex_jacobians_match_finite_differences(kind):
    rng = np.random.default_rng(20 + kind)
    for _ in range(20):
        qa = _rand_quat(rng)
        # neighbour within 60 deg so that the double-cover flip is not crossed
        qb = _perturb_rot(qa, rng.normal(size=3) * 0.4)
        s = rng.uniform(0.6, 1.4)
        la, lb = rng.uniform(0.3, 1.5, 2)
        ob = rng.normal(size=3)
        r = oracle.vertex_constraint(kind, qa, qb, s, la, lb, ob)
        eps = 1e-6

        def C_of(qa_=qa, qb_=qb, s_=s):
            return oracle.vertex_constraint(kind, qa_, qb_, s_, la, lb, ob)["C"]

        for c in range(3):
            e = np.zeros(3); e[c] = eps
            fd = (C_of(qa_=_perturb_rot(qa, e)) - C_of(qa_=_perturb_rot(qa, -e))) / (2 * eps)
            np.testing.assert_allclose(r["Jtha"][:, c], fd, rtol=1e-6, atol=1e-7)
            fd = (C_of(qb_=_perturb_rot(qb, e)) - C_of(qb_=_perturb_rot(qb, -e))) / (2 * eps)
            np.testing.assert_allclose(r["Jthb"][:, c], fd, rtol=1e-6, atol=1e-7)
        fd = (C_of(s_=s + eps) - C_of(s_=s - eps)) / (2 * eps)
        np.testing.assert_allclose(r["Js"], fd, rtol=1e-6, atol=1e-7)


# --------------------------------------------------------------------------
# Constraint values vs independent closed forms
# --------------------------------------------------------------------------

def test_stretch_value_is_strain_along_tangent():
    q = S.quat_from_z(np.array([0.3, -0.4, 0.866]))
    d3 = _rot(q, [0, 0, 1])
    for lam in (0.7, 1.0, 1.3):
        r = oracle.segment_constraint(0, np.zeros(3), lam * 0.5 * d3, 1, 1, q, 0.5)
        np.testing.assert_allclose(r["C"], (lam - 1) * d3, atol=1e-14)


def _deformation_det(c0, c1, s0, s1, q, lbar, x=0.0, y=0.0):
    """det of the Jacobian of p(x, y, z) = c(z) + s(z) R q_disc (Eq. deformed
    parametrization) at the segment midpoint, by central differences of the
    parametrisation itself (c, s linear along the element, R constant)."""
    R = np.stack([_rot(q, e) for e in np.eye(3)], axis=1)

    def p(xx, yy, z):
        t = z / lbar
        c = (1 - t) * c0 + t * c1
        s = (1 - t) * s0 + t * s1
        return c + s * R @ np.array([xx, yy, 0.0])

    h = 1e-6
    z = 0.5 * lbar
    J = np.stack([(p(x + h, y, z) - p(x - h, y, z)) / (2 * h),
                  (p(x, y + h, z) - p(x, y - h, z)) / (2 * h),
                  (p(x, y, z + h) - p(x, y, z - h)) / (2 * h)], axis=1)
    return np.linalg.det(J)


def test_volume_value_is_deformation_determinant():
    """C_V + 1 = |grad p| at the disc centre (App. A determinant), rest det = 1."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        q = _rand_quat(rng)
        d3 = _rot(q, [0, 0, 1])
        lbar = rng.uniform(0.2, 1.0)
        c0 = rng.normal(size=3)
        c1 = c0 + lbar * rng.uniform(0.5, 1.5) * (d3 + 0.2 * rng.normal(size=3))
        s0, s1 = rng.uniform(0.6, 1.4, 2)
        det = _deformation_det(c0, c1, s0, s1, q, lbar)
        # the oracle's V uses the midpoint scale; at the midpoint s(z) = s_m
        r = oracle.segment_constraint(1, c0, c1, s0, s1, q, lbar)
        np.testing.assert_allclose(r["C"][0] + 1.0, det, rtol=1e-7)


def test_vector_volume_form():
    """The printed vector volume term (Sec. 5, App. A): its component along d3
    is the determinant's scalar form; it vanishes on a volume-preserving
    stretch along the frame (s = 1/sqrt(lambda)) where stretch alone does not;
    unlike the scalar form it also measures shear across the frame."""
    rng = np.random.default_rng(31)
    for _ in range(20):
        q = _rand_quat(rng)
        d3 = _rot(q, [0, 0, 1])
        lbar = rng.uniform(0.2, 1.0)
        c0 = rng.normal(size=3)
        c1 = c0 + lbar * rng.uniform(0.5, 1.5) * (d3 + 0.3 * rng.normal(size=3))
        s0, s1 = rng.uniform(0.6, 1.4, 2)
        cv = oracle.segment_constraint(4, c0, c1, s0, s1, q, lbar)["C"]
        cs = oracle.segment_constraint(1, c0, c1, s0, s1, q, lbar)["C"][0]
        np.testing.assert_allclose(cv @ d3, cs, rtol=1e-12, atol=1e-12)
        lam = rng.uniform(0.5, 2.0)
        s = 1.0 / math.sqrt(lam)
        cv = oracle.segment_constraint(4, c0, c0 + lam * lbar * d3, s, s, q, lbar)["C"]
        np.testing.assert_allclose(cv, 0.0, atol=1e-12)
        e1 = _rot(q, [1, 0, 0])
        gam = rng.uniform(0.05, 0.5)
        cv = oracle.segment_constraint(4, c0, c0 + lbar * (d3 + gam * e1), 1.0, 1.0, q, lbar)["C"]
        cs = oracle.segment_constraint(1, c0, c0 + lbar * (d3 + gam * e1), 1.0, 1.0, q, lbar)["C"][0]
        np.testing.assert_allclose(cv, gam * e1, atol=1e-12)
        assert abs(cs) < 1e-12


def test_darboux_of_uniform_twist_and_bend():
    """Omega = 4/(la+lb) Im(conj(qa) qb): rotating by phi about the body axis k
    gives Omega = (2/l) sin(phi/2) e_k (Sec. 7.5)."""
    l = 0.02
    qa = S.quat_from_z(np.array([1.0, 2.0, -0.5]))
    for k in range(3):
        for phi in (0.01, 0.3, 1.2):
            axis_world = _rot(qa, np.eye(3)[k])
            qb = _perturb_rot(qa, phi * axis_world)
            r = oracle.vertex_constraint(0, qa, qb, 1.0, l, l, np.zeros(3))
            expect = np.zeros(3)
            expect[k] = 2.0 / l * math.sin(phi / 2)
            np.testing.assert_allclose(r["C"], expect, atol=1e-10)


# --------------------------------------------------------------------------
# Stiffness constants vs quadrature of the paper's disc integrands
# --------------------------------------------------------------------------

def _disc_quadrature(r, n=64):
    """Gauss-Legendre in radius x uniform in angle; nodes (x, y) and weights."""
    gx, gw = np.polynomial.legendre.leggauss(n)
    rho = 0.5 * r * (gx + 1)
    wr = 0.5 * r * gw * rho
    th = np.linspace(0, 2 * np.pi, 2 * n, endpoint=False)
    wt = 2 * np.pi / (2 * n)
    R, T = np.meshgrid(rho, th, indexing="ij")
    W = np.outer(wr, np.full(th.size, wt))
    return R * np.cos(T), R * np.sin(T), W


def _one_rod_scene(n=4, r=0.03, lbar=0.01, cs=1e-6, cb=2e-6, cv=3e-6, rho=1000.0):
    off = np.array([0, n], np.int32)
    pos = np.zeros((n, 3)); pos[:, 0] = np.arange(n) * lbar
    q = np.tile(S.quat_from_z(np.array([1.0, 0, 0])), (n - 1, 1))
    return S.Scene(
        name="one", rod_offsets=off, rest_pos=pos, rest_quat=q, radius=np.full(n, r),
        density=np.array([rho]), c_stretch=np.array([cs]), c_bend=np.array([cb]),
        c_volume=np.array([cv]), group=np.zeros(1, np.int32), gravity=np.zeros(3),
        pin_vertex=np.zeros(0, np.int32), pin_bone=np.zeros(0, np.int32),
        pin_offset=np.zeros((0, 3)), bones=None, planes=np.zeros((0, 4)),
        contact_compliance=1e-9, contacts=False, volume=True, dt=1 / 60, substeps=1,
        iterations=1, frames=1)


def test_compliances_equal_integrated_energy_coefficients():
    """K (= 1/alpha) per unit length equals the disc integral of the strain /
    volume energy densities of Sec. 5 for a unit constraint violation, with the
    1/2 ||W||_K^2 convention of Eq. variational_implicit."""
    r, l = 0.03, 0.01
    cs, cb, cv = 1e-6, 2e-6, 3e-6
    ks, kb, kv = 1 / cs, 1 / cb, 1 / cv
    sc = _one_rod_scene(r=r, lbar=l, cs=cs, cb=cb, cv=cv)
    o = oracle.OracleScene(sc)
    X, Y, W = _disc_quadrature(r)
    area = W.sum()
    np.testing.assert_allclose(area, math.pi * r * r, rtol=1e-12)
    # strain energy density ||R^T grad p - Rbar^T grad pbar||_K^2 with K = k I
    # (App. A): a unit stretch of grad c along d3 -> integrand k * 1
    K_S = (ks * W).sum()
    # cross-section scale (s - sbar) = 1 enters the xx and yy entries -> (kx + ky)
    K_X = (2 * ks * W).sum()
    # scale gradient: entries (grad s x, grad s y) in the third column
    K_G = (ks * (X ** 2 + Y ** 2) * W).sum()
    # bend/twist: ||(delta Omega) x q||_K^2 for unit delta along u, v, w
    def bend(delta):
        cr = np.stack([-delta[2] * Y, delta[2] * X, delta[0] * Y - delta[1] * X])
        return (kb * (cr ** 2).sum(axis=0) * W).sum()
    K_B = [bend(e) for e in np.eye(3)]
    # volume: |grad p| - 1 for the determinant s^2 d3.grad c + s^3 (Om_u y - Om_v x)
    K_V = (kv * W).sum()
    K_Vb = (kv * Y ** 2 * W).sum()  # unit Omega_u
    a = o.segment_compliance(1)
    np.testing.assert_allclose(1 / (a[0] * l), K_S, rtol=1e-10)
    np.testing.assert_allclose(1 / (a[1] * l), K_V, rtol=1e-10)
    np.testing.assert_allclose(1 / (a[2] * l), K_X, rtol=1e-10)
    np.testing.assert_allclose(1 / (a[3] * l), K_G, rtol=1e-10)
    b = o.vertex_compliance(1)
    np.testing.assert_allclose(1 / (b[:3] * l), K_B, rtol=1e-10)
    np.testing.assert_allclose(1 / (b[3] * l), K_Vb, rtol=1e-10)


def test_lumped_inertias_sum_to_rod_totals():
    """Position weights sum to the rod mass sum(pi r^2 rho l), scale weights to
    sum(pi r^4 rho l / 2) (App. B inertia integrals)."""
    sc = S.muscle_rig(n_rods=3, mesh_verts=0)
    sc = dataclasses.replace(sc, pin_vertex=np.zeros(0, np.int32), pin_bone=np.zeros(0, np.int32),
                             pin_offset=np.zeros((0, 3)))
    o = oracle.OracleScene(sc)
    lb, _ = o.rest()
    for r in range(sc.n_rods):
        v0, v1 = sc.rod_offsets[r], sc.rod_offsets[r + 1]
        m = s_ = 0.0
        for i in range(v0, v1):
            mi, si = o.vertex_inverse_inertia(i)
            m += 1 / mi
            s_ += 1 / si
        rm = 0.5 * (sc.radius[v0:v1 - 1] + sc.radius[v0 + 1:v1])
        l = lb[v0 - r:v1 - 1 - r]
        np.testing.assert_allclose(m, (math.pi * rm ** 2 * 1000 * l).sum(), rtol=1e-12)
        np.testing.assert_allclose(s_, (math.pi * rm ** 4 * 1000 * l / 2).sum(), rtol=1e-12)


# --------------------------------------------------------------------------
# whole steps: rest, free fall, rigid motion, momentum, unit quaternions
# --------------------------------------------------------------------------

def _helix_scene(n_rods=4, n=12, lbar=0.01, seed=5):
    """Rods whose rest shape is a helix with frames aligned to the tangents and
    twisted about them, so that every rest Darboux component is non-zero."""
    rng = np.random.default_rng(seed)
    off = np.arange(n_rods + 1, dtype=np.int32) * n
    pos, quat = [], []
    for r in range(n_rods):
        t = np.arange(n) * 0.35
        p = np.stack([0.02 * np.cos(t), 0.02 * np.sin(t), 0.01 * t], 1) + np.array([0.2 * r, 0, 0])
        d = np.diff(p, axis=0)
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        q = S.quat_from_z(d)
        tw = rng.uniform(-0.4, 0.4, n - 1)
        q = S.quat_mul(S.axis_angle_quat(d * tw[:, None]), q)
        pos.append(p)
        quat.append(q)
    pos = np.concatenate(pos)
    return S.Scene(
        name="helix", rod_offsets=off, rest_pos=pos, rest_quat=np.concatenate(quat),
        radius=rng.uniform(0.004, 0.01, n_rods * n), density=np.full(n_rods, 1000.0),
        c_stretch=np.full(n_rods, 1e-6), c_bend=np.full(n_rods, 1e-6), c_volume=np.full(n_rods, 1e-6),
        group=np.arange(n_rods, dtype=np.int32), gravity=np.zeros(3),
        pin_vertex=np.zeros(0, np.int32), pin_bone=np.zeros(0, np.int32), pin_offset=np.zeros((0, 3)),
        bones=None, planes=np.zeros((0, 4)), contact_compliance=1e-9, contacts=False, volume=True,
        dt=1 / 60, substeps=10, iterations=4, frames=1)


@pytest.mark.parametrize("jacobi", [False, True], ids=["colours", "jacobi"])
def test_rest_state_is_stationary_without_gravity(jacobi):
    sc = dataclasses.replace(_helix_scene(), jacobi=jacobi)
    o = oracle.OracleScene(sc)
    _, ob = o.rest()
    assert np.abs(ob).max() > 1.0  # curved and twisted: Omega_bar is not zero
    x0 = o.get_state()
    rms = o.constraint_rms()
    assert max(rms.values()) < 1e-13
    for _ in range(3):
        assert o.step() == 0
    x1 = o.get_state()
    np.testing.assert_allclose(x1["x"], x0["x"], atol=1e-12)
    np.testing.assert_allclose(x1["s"], x0["s"], atol=1e-12)
    np.testing.assert_allclose(np.abs((x1["q"] * x0["q"]).sum(1)), 1.0, atol=1e-12)
    np.testing.assert_allclose(x1["v"], 0.0, atol=1e-10)


def test_free_fall_matches_discrete_closed_form():
    """Unpinned rod at rest under gravity: constraints stay satisfied, every
    vertex follows x_n = x_0 + n h v_0 + g h^2 n (n+1)/2 (the prediction /
    velocity update sequence), and velocity v_n = v_0 + n h g."""
    sc = dataclasses.replace(S.plain_small(n_rods=3), pin_vertex=np.zeros(0, np.int32),
                             pin_bone=np.zeros(0, np.int32), pin_offset=np.zeros((0, 3)))
    o = oracle.OracleScene(sc)
    v0 = np.array([0.3, 0.1, -0.2])
    st = o.get_state()
    o.set_state(v=np.tile(v0, (sc.nv, 1)))
    frames = 3
    for _ in range(frames):
        assert o.step() == 0
    n = frames * sc.substeps
    h = sc.dt / sc.substeps
    expect = st["x"] + n * h * v0 + sc.gravity * h * h * n * (n + 1) / 2
    out = o.get_state()
    np.testing.assert_allclose(out["x"], expect, atol=1e-12)
    np.testing.assert_allclose(out["v"], np.tile(v0 + n * h * sc.gravity, (sc.nv, 1)), atol=1e-10)


def test_twist_spin_decay_closed_form():
    """A two-vertex rod spinning about its own axis has only the spin DOF free:
    the prediction rotates by 2 atan(h w / 2) per substep and the velocity
    update returns w / sqrt(1 + (h w / 2)^2)."""
    sc = _one_rod_scene(n=2)
    o = oracle.OracleScene(sc)
    st = o.get_state()
    d3 = _rot(st["q"][0], [0, 0, 1])
    w = 7.0
    o.set_state(w=(w * d3)[None, :])
    h = sc.dt
    ang = 0.0
    wn = w
    for _ in range(5):
        assert o.step(dt=h, substeps=1, iterations=2) == 0
        ang += 2 * math.atan(h * wn / 2)
        wn = wn / math.sqrt(1 + (h * wn / 2) ** 2)
    out = o.get_state()
    qexp = _perturb_rot(st["q"][0], ang * d3)
    assert abs(abs(np.dot(out["q"][0], qexp)) - 1) < 1e-12
    np.testing.assert_allclose(out["w"][0], wn * d3, atol=1e-9)


def _rigid(R, t, x):
    return x @ R.T + t


@pytest.mark.parametrize("jacobi", [False, True], ids=["colours", "jacobi"])
def test_rigid_motion_invariance(jacobi):
    """Rotating and translating the whole scene (rest pose, initial state,
    pins and gravity) rotates and translates the result."""
    rng = np.random.default_rng(7)
    base = dataclasses.replace(S.plain_small(n_rods=4, n_verts=12), jacobi=jacobi)
    # start from a perturbed state so that every constraint family is active
    init_q = S.quat_mul(S.axis_angle_quat(rng.normal(size=(base.ns, 3)) * 0.2), base.rest_quat)
    init_x = base.rest_pos + rng.normal(size=base.rest_pos.shape) * 1e-3
    qR = _rand_quat(rng)
    R = np.stack([_rot(qR, e) for e in np.eye(3)], axis=1)
    t = np.array([0.3, -1.0, 2.0])
    rot = dataclasses.replace(
        base, rest_pos=_rigid(R, t, base.rest_pos),
        rest_quat=S.quat_mul(np.tile(qR, (base.ns, 1)), base.rest_quat),
        gravity=R @ base.gravity, pin_offset=_rigid(R, t, base.pin_offset))
    o1 = oracle.OracleScene(base)
    o2 = oracle.OracleScene(rot)
    o1.set_state(x=init_x, q=init_q)
    o2.set_state(x=_rigid(R, t, init_x), q=S.quat_mul(np.tile(qR, (base.ns, 1)), init_q))
    for _ in range(3):
        assert o1.step() == 0 and o2.step() == 0
    a, b = o1.get_state(), o2.get_state()
    np.testing.assert_allclose(b["x"], _rigid(R, t, a["x"]), atol=1e-11)
    np.testing.assert_allclose(b["s"], a["s"], atol=1e-11)
    qa = S.quat_mul(np.tile(qR, (base.ns, 1)), a["q"])
    np.testing.assert_allclose(np.abs((qa * b["q"]).sum(1)), 1.0, atol=1e-11)
    np.testing.assert_allclose(b["w"], a["w"] @ R.T, atol=1e-8)


def test_linear_momentum_conserved_without_external_forces():
    rng = np.random.default_rng(8)
    sc = dataclasses.replace(S.muscle_rig(n_rods=6, mesh_verts=0), gravity=np.zeros(3),
                             pin_vertex=np.zeros(0, np.int32), pin_bone=np.zeros(0, np.int32),
                             pin_offset=np.zeros((0, 3)), contacts=False)
    o = oracle.OracleScene(sc)
    st = o.get_state()
    o.set_state(x=st["x"] + rng.normal(size=st["x"].shape) * 2e-3,
                q=S.quat_mul(S.axis_angle_quat(rng.normal(size=(sc.ns, 3)) * 0.3), st["q"]),
                v=rng.normal(size=st["x"].shape) * 0.1, sdot=rng.normal(size=sc.nv) * 0.1)
    m = np.array([1 / o.vertex_inverse_inertia(i)[0] for i in range(sc.nv)])
    p0 = (m[:, None] * o.get_state()["v"]).sum(0)
    for _ in range(3):
        assert o.step() == 0
    p1 = (m[:, None] * o.get_state()["v"]).sum(0)
    np.testing.assert_allclose(p1, p0, atol=1e-12 * max(1.0, np.abs(p0).max()))


# --------------------------------------------------------------------------
# how the solve uses compliance and inertia (Sec. 6 "Correction steps",
# App. B, App. C): static and dynamic closed forms
# --------------------------------------------------------------------------

def _straight_rod(n, lbar, r, cs, cb, rho, direction, pins, gravity):
    """One straight rod of n vertices along `direction`, volume term off (the
    scales then stay at one), vertices `pins` held at their rest positions."""
    d = np.asarray(direction, float)
    d = d / np.linalg.norm(d)
    pos = np.arange(n)[:, None] * lbar * d[None, :]
    pins = np.asarray(pins, np.int32)
    return S.Scene(
        name="straight", rod_offsets=np.array([0, n], np.int32), rest_pos=pos,
        rest_quat=np.tile(S.quat_from_z(d), (n - 1, 1)), radius=np.full(n, r), density=np.array([rho]),
        c_stretch=np.array([cs]), c_bend=np.array([cb]), c_volume=np.array([cs]), group=np.zeros(1, np.int32),
        gravity=np.asarray(gravity, float), pin_vertex=pins, pin_bone=np.full(len(pins), -1, np.int32),
        pin_offset=pos[pins], bones=None, planes=np.zeros((0, 4)), contact_compliance=1e-9, contacts=False,
        volume=False, dt=1 / 60, substeps=1, iterations=1, frames=1)


def test_hanging_rod_strain_is_weight_over_stiffness():
    """Hooke's law in the solve's static limit.  A vertical rod hangs from its
    pinned top vertex.  Stepping with the velocities cleared after every step
    (and a fully converged inner solve) drives the state to the minimum of
    elastic plus gravitational energy.  Segment j then carries the weight of
    the lumped vertex masses below it: strain_j = g W_j c_s / (pi r^2), the
    stress over the modulus 1/c_s.  Only a compliance that enters the update as
    alpha / h^2 reaches this equilibrium (alpha / h would stiffen the rod by a
    factor 1/h)."""
    n, lbar, r, cs, rho, g = 8, 0.02, 0.01, 1e-6, 1000.0, 9.81
    sc = _straight_rod(n, lbar, r, cs, 1e-6, rho, [0, -1, 0], [0], [0, -g, 0])
    o = oracle.OracleScene(sc)
    for _ in range(300):
        assert o.step(dt=1 / 60, substeps=1, iterations=1000) == 0
        o.set_state(v=np.zeros((n, 3)), sdot=np.zeros(n), w=np.zeros((n - 1, 3)))
    x = o.get_state()["x"]
    strain = np.linalg.norm(np.diff(x, axis=0), axis=1) / lbar - 1
    M = math.pi * r * r * rho * lbar  # segment mass; vertices carry half of each adjacent segment
    m = np.full(n, M)
    m[0] = m[-1] = 0.5 * M
    W = np.array([m[j + 1:].sum() for j in range(n - 1)])
    expect = g * W * cs / (math.pi * r * r)
    np.testing.assert_allclose(strain, expect, rtol=1e-4)


def _zero_crossings(sig, h):
    t = []
    for k in range(1, len(sig)):
        if (sig[k - 1] < 0) != (sig[k] < 0):
            t.append(h * (k - 1 + sig[k - 1] / (sig[k - 1] - sig[k])))
    return np.array(t)


def test_twist_oscillation_frequency():
    """Torsional mode of two segments between three pinned vertices.  The
    twist part of the bend/twist term stores (pi r^4 / (2 c_b l)) phi^2 / 2 for a
    relative twist phi, and each segment spins about its axis with inertia
    M r^2 / 2 (App. B: s^2 m I with I_zz = pi r^4 / 2), so counter-rotating
    segments oscillate at w = sqrt(2 / (c_b rho)) / l.  The solve is an
    implicit step, whose phase advances by atan(w h) per step: the measured
    frequency must be atan(w h) / h.  A factor in the compliance scaling, the
    twist stiffness or the axial inertia moves it far outside the bound."""
    lbar, r, cb, rho = 0.05, 0.01, 1e-5, 1000.0
    sc = _straight_rod(3, lbar, r, 1e-8, cb, rho, [1, 0, 0], [0, 1, 2], np.zeros(3))
    o = oracle.OracleScene(sc)
    o.set_state(w=np.array([[-2.0, 0, 0], [2.0, 0, 0]]))
    h = 1 / 6000
    sig = []
    for _ in range(400):
        assert o.step(dt=h, substeps=1, iterations=4) == 0
        q = o.get_state()["q"]
        p = S.quat_mul(q[0] * np.array([-1, -1, -1, 1]), q[1])  # conj(q0) q1: twist about the rod axis
        sig.append(2 * math.atan2(p[2], p[3]))
    tc = _zero_crossings(np.array(sig), h)
    assert len(tc) >= 4
    w = math.sqrt(2 / (cb * rho)) / lbar
    np.testing.assert_allclose(math.pi / np.diff(tc).mean(), math.atan(w * h) / h, rtol=5e-5)


def test_shear_rocking_frequency():
    """A single segment between two pinned vertices, turned about an axis
    across it: the stretch/shear term C = dx / l - d3 stores
    (pi r^2 l / c_s) psi^2 / 2 for a tilt psi, against the transverse inertia
    M r^2 / 4, so it rocks at w = sqrt(4 / (c_s rho r^2)); the implicit step
    advances atan(w h) per step."""
    lbar, r, cs, rho = 0.05, 0.05, 1e-4, 1000.0
    sc = _straight_rod(2, lbar, r, cs, 1e-5, rho, [1, 0, 0], [0, 1], np.zeros(3))
    o = oracle.OracleScene(sc)
    o.set_state(w=np.array([[0, 0.5, 0]]))
    w = math.sqrt(4 / (cs * rho * r * r))
    h = 2 * math.pi / w / 200
    sig = []
    for _ in range(800):
        assert o.step(dt=h, substeps=1, iterations=4) == 0
        d3 = S.quat_rotate(o.get_state()["q"][0], np.array([0, 0, 1.0]))
        sig.append(math.atan2(-d3[2], d3[0]))
    tc = _zero_crossings(np.array(sig), h)
    assert len(tc) >= 6
    np.testing.assert_allclose(math.pi / np.diff(tc).mean(), math.atan(w * h) / h, rtol=5e-5)


def _planar_scene(n_rods=3, n=6, lbar=0.01, r=0.012, seed=5):
    """Rods curved in the xy-plane (rest frames from the tangents, so one
    frame axis is +-z): planar motion stays planar."""
    rng = np.random.default_rng(seed)
    pos, quat = [], []
    for k in range(n_rods):
        ang = np.cumsum(np.r_[rng.uniform(0, 2 * math.pi), rng.uniform(-0.5, 0.5, n - 2)])
        d = np.stack([np.cos(ang), np.sin(ang), np.zeros(n - 1)], 1)
        pos.append(np.vstack([np.zeros(3), np.cumsum(lbar * d, 0)]) + np.array([0.04 * k, 0.01 * k, 0]))
        quat.append(S.quat_from_z(d))
    return S.Scene(
        name="planar", rod_offsets=np.arange(n_rods + 1, dtype=np.int32) * n, rest_pos=np.concatenate(pos),
        rest_quat=np.concatenate(quat), radius=np.full(n_rods * n, r), density=np.full(n_rods, 1000.0),
        c_stretch=np.full(n_rods, 1e-6), c_bend=np.full(n_rods, 1e-6), c_volume=np.full(n_rods, 1e-6),
        group=np.arange(n_rods, dtype=np.int32), gravity=np.zeros(3),
        pin_vertex=np.zeros(0, np.int32), pin_bone=np.zeros(0, np.int32), pin_offset=np.zeros((0, 3)),
        bones=None, planes=np.zeros((0, 4)), contact_compliance=1e-9, contacts=False, volume=True,
        dt=1 / 60, substeps=10, iterations=4, frames=1)


def _angular_momentum(sc, st):
    """sum m_i x_i x v_i + sum_j I_j w_j with the closed-form inertias: vertex
    masses lumped from M_j = pi r_m^2 rho l_j, segment inertia
    s_m^2 R diag(M r_m^2 / 4, M r_m^2 / 4, M r_m^2 / 2) R^T (App. B)."""
    x, v, q, w, s = st["x"], st["v"], st["q"], st["w"], st["s"]
    L = np.zeros(3)
    g = 0
    for r in range(sc.n_rods):
        for j in range(sc.rod_offsets[r], sc.rod_offsets[r + 1] - 1):
            lj = np.linalg.norm(sc.rest_pos[j + 1] - sc.rest_pos[j])
            rm = 0.5 * (sc.radius[j] + sc.radius[j + 1])
            Mj = math.pi * rm * rm * sc.density[r] * lj
            L += 0.5 * Mj * (np.cross(x[j], v[j]) + np.cross(x[j + 1], v[j + 1]))
            R = np.stack([S.quat_rotate(q[g], e) for e in np.eye(3)], 1)
            sm = 0.5 * (s[j] + s[j + 1])
            I = sm * sm * Mj * rm * rm * (R @ np.diag([0.25, 0.25, 0.5]) @ R.T)
            L += I @ w[g]
            g += 1
    return L


def test_angular_momentum_conserved_in_planar_motion():
    """Without gravity, pins or contacts every constraint is invariant under
    rotations, so each update changes sum m x dx + sum I dtheta by zero: the
    angular momentum counted with the closed-form inertias is conserved.  The
    motion is kept planar (velocities in the plane, spins about its normal, a
    principal axis of every segment), because the paper's prediction carries
    the angular velocity without a gyroscopic term and so does not conserve
    the momentum of spins about non-principal axes.  Counting the spin with
    half or twice the transverse inertia breaks the balance by > 15 %."""
    sc = _planar_scene()
    o = oracle.OracleScene(sc)
    rng = np.random.default_rng(3)
    st = o.get_state()
    v = rng.normal(scale=0.02, size=st["v"].shape)
    v[:, 2] = 0
    w = np.zeros(st["w"].shape)
    w[:, 2] = rng.normal(scale=5.0, size=len(w))
    o.set_state(v=v, w=w)
    L0 = _angular_momentum(sc, o.get_state())
    spin0 = L0 - _angular_momentum(sc, dict(o.get_state(), w=np.zeros_like(w)))
    assert np.linalg.norm(spin0) > 0.2 * np.linalg.norm(L0)  # the spins carry a real share
    for _ in range(10):
        assert o.step() == 0
    L1 = _angular_momentum(sc, o.get_state())
    assert np.linalg.norm(L1 - L0) < 1e-3 * np.linalg.norm(L0)

def test_contact_conserves_momentum_and_separates():
    """Two crossing two-vertex rods driven into each other (g = 0, no pins):
    the contact keeps total momentum and leaves the pills non-penetrating."""
    off = np.array([0, 2, 4], np.int32)
    pos = np.array([[-0.1, 0, 0], [0.1, 0, 0], [0, -0.1, 0.05], [0, 0.1, 0.05]], float)
    q = np.stack([S.quat_from_z(np.array([1.0, 0, 0])), S.quat_from_z(np.array([0, 1.0, 0]))])
    sc = S.Scene(name="x", rod_offsets=off, rest_pos=pos, rest_quat=q, radius=np.full(4, 0.02),
                 density=np.full(2, 1000.0), c_stretch=np.full(2, 1e-7), c_bend=np.full(2, 1e-7),
                 c_volume=np.full(2, 1e-7), group=np.array([0, 1], np.int32), gravity=np.zeros(3),
                 pin_vertex=np.zeros(0, np.int32), pin_bone=np.zeros(0, np.int32),
                 pin_offset=np.zeros((0, 3)), bones=None, planes=np.zeros((0, 4)),
                 contact_compliance=1e-9, contacts=True, volume=True, dt=1 / 60, substeps=10,
                 iterations=4, frames=1)
    o = oracle.OracleScene(sc)
    v = np.zeros((4, 3)); v[2:, 2] = -3.0
    o.set_state(v=v)
    m = np.array([1 / o.vertex_inverse_inertia(i)[0] for i in range(4)])
    p0 = (m[:, None] * v).sum(0)
    touched = False
    smin = 1.0
    for _ in range(30):
        assert o.step(dt=sc.dt / 10, substeps=1) == 0
        touched |= o.last_pairs().shape[0] > 0
        smin = min(smin, o.get_state()["s"].min())
    # contacts act on radii too: pinched rods get thinner (App. E, Bergou comparison)
    assert smin < 0.999
    st = o.get_state()
    np.testing.assert_allclose((m[:, None] * st["v"]).sum(0), p0, atol=1e-12)
    assert touched
    rad = st["s"] * 0.02
    a, b, C = oracle.narrowphase(st["x"][0], rad[0], st["x"][1], rad[1], st["x"][2], rad[2],
                                 st["x"][3], rad[3])
    assert C > -1e-3 * 0.02


def test_quaternions_stay_unit():
    sc = S.batching(n_rods=20)
    o = oracle.OracleScene(sc)
    for _ in range(2):
        assert o.step() == 0
    q = o.get_state()["q"]
    np.testing.assert_allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-12)


@pytest.mark.parametrize("vector_form", [False, True], ids=["scalar", "vector"])
def test_volume_held_and_rod_thins_when_stretched(vector_form):
    """A rod pinned at both ends at 1.3x its rest length (E1, E8).  With a stiff
    volume term and enough iterations the solver reaches the closed form
    s = 1/sqrt(1.3) (segment volume = rest volume); softer volume compliance
    leaves a larger volume error; without the volume term s stays at 1 and the
    volume grows by the stretch (30 %)."""
    def run(cv, iters=100, volume=True):
        n = 10
        sc = _one_rod_scene(n=n, r=0.01, lbar=0.01, cs=1e-5, cb=1e-5, cv=cv)
        sc = dataclasses.replace(sc, volume=volume, volume_vector=vector_form,
                                 pin_vertex=np.array([0, n - 1], np.int32),
                                 pin_bone=np.array([-1, -1], np.int32),
                                 pin_offset=np.array([[0, 0, 0], [1.3 * 0.01 * (n - 1), 0, 0]]))
        o = oracle.OracleScene(sc)
        st = o.get_state()
        o.set_state(x=st["x"] * np.array([1.3, 1.0, 1.0]))
        for _ in range(10):
            assert o.step(substeps=10, iterations=iters) == 0
        st = o.get_state()
        seg = np.linalg.norm(np.diff(st["x"], axis=0), axis=1)
        sm = 0.5 * (st["s"][1:] + st["s"][:-1])
        return np.abs(sm ** 2 * seg / 0.01 - 1).max(), sm
    err_stiff, s = run(1e-9)
    err_mid, _ = run(1e-6)
    err_soft, _ = run(1e-4)
    err_off, s_off = run(1e-9, volume=False)
    assert err_stiff < 1e-4
    np.testing.assert_allclose(s, 1 / math.sqrt(1.3), atol=5e-4)
    assert err_stiff < err_mid < err_soft < err_off
    np.testing.assert_allclose(err_off, 0.3, atol=2e-3)
    np.testing.assert_allclose(s_off, 1.0, atol=1e-3)


def test_solver_converges_on_instantaneous_stretch():
    """E9-style: bars pulled to 2x; the stretch residual falls as iterations grow."""
    n = 12
    sc = _one_rod_scene(n=n, r=0.01, lbar=0.01, cs=1e-9, cb=1e-7, cv=1e-9)
    sc = dataclasses.replace(sc, pin_vertex=np.array([0, n - 1], np.int32), pin_bone=np.array([-1, -1], np.int32),
                             pin_offset=np.array([[0, 0, 0], [2.0 * 0.01 * (n - 1), 0, 0]]))
    res = []
    for iters in (1, 4, 16, 64):
        o = oracle.OracleScene(sc)
        assert o.step(dt=1 / 60, substeps=1, iterations=iters) == 0
        res.append(o.constraint_rms()["S"])
    assert res[0] > res[1] > res[2] > res[3]


# --------------------------------------------------------------------------
# collision geometry: projection, narrowphase, half-planes, broadphase
# --------------------------------------------------------------------------

def _capsule_sd(c1, r1, c2, r2, x, n=200001):
    t = np.linspace(0, 1, n)
    c = c1[None, :] + t[:, None] * (c2 - c1)[None, :]
    r = r1 + t * (r2 - r1)
    f = np.linalg.norm(x[None, :] - c, axis=1) - r
    k = np.argmin(f)
    return t[k], f[k]


def test_pill_projection_matches_dense_sampling():
    rng = np.random.default_rng(11)
    for _ in range(200):
        c1, c2 = rng.normal(size=3), rng.normal(size=3)
        l = np.linalg.norm(c2 - c1)
        r1, r2 = rng.uniform(0.05, 0.6 * l, 2)
        x = rng.normal(size=3) * 2
        t = oracle.pill_project(c1, r1, c2, r2, x)
        ts, fs = _capsule_sd(c1, r1, c2, r2, x)
        ct = c1 + t * (c2 - c1)
        f = np.linalg.norm(x - ct) - (r1 + t * (r2 - r1))
        assert f <= fs + 1e-9
        assert abs(f - fs) < 1e-8


def test_narrowphase_matches_dense_scan():
    """The 10-step dichotomous search reaches the minimum of Eq. collsearch to
    within what a 2^-10 bracket allows."""
    rng = np.random.default_rng(12)
    for _ in range(60):
        a1 = rng.normal(size=3); a2 = a1 + rng.normal(size=3)
        b1 = rng.normal(size=3) * 0.5; b2 = b1 + rng.normal(size=3)
        ra = rng.uniform(0.05, 0.3, 2); rb = rng.uniform(0.05, 0.3, 2)
        al, be, C = oracle.narrowphase(a1, ra[0], a2, ra[1], b1, rb[0], b2, rb[1])
        alphas = np.linspace(0, 1, 2001)
        P = a1[None, :] + alphas[:, None] * (a2 - a1)[None, :]
        t = np.linspace(0, 1, 2001)
        cb = b1[None, :] + t[:, None] * (b2 - b1)[None, :]
        rbt = rb[0] + t * (rb[1] - rb[0])
        sd = (np.linalg.norm(P[:, None, :] - cb[None, :, :], axis=2) - rbt[None, :]).min(axis=1)
        fs = sd - (ra[0] + alphas * (ra[1] - ra[0]))
        lip = np.linalg.norm(a2 - a1) + abs(ra[1] - ra[0])
        assert C <= fs.min() + lip * 2e-3 + 1e-6
        assert C >= fs.min() - 1e-6


def test_half_plane_holds_pill_above_floor():
    """A falling rod lands on a floor half-plane: after settling no point of any
    pill is below the plane (checked by dense sampling of the capsules)."""
    sc = dataclasses.replace(_one_rod_scene(n=6, r=0.01, lbar=0.02),
                             gravity=np.array([0, -9.81, 0]),
                             planes=np.array([[0.0, 1.0, 0.0, -0.05]]))
    o = oracle.OracleScene(sc)
    st = o.get_state()
    o.set_state(q=S.quat_mul(np.tile(S.axis_angle_quat(np.array([0, 0, 0.3])), (sc.ns, 1)), st["q"]))
    for _ in range(40):
        assert o.step() == 0
    st = o.get_state()
    rad = st["s"] * 0.01
    # resting contact squeezes the radius of the vertices that touch the floor
    low = np.argmin(st["x"][:, 1])
    assert st["s"][low] < 1.0
    for j in range(sc.ns):
        t = np.linspace(0, 1, 1001)
        y = (1 - t) * st["x"][j, 1] + t * st["x"][j + 1, 1] - ((1 - t) * rad[j] + t * rad[j + 1])
        assert y.min() > -0.05 - 2e-4


def test_broadphase_grid_equals_brute_force():
    rng = np.random.default_rng(13)
    for trial in range(6):
        n_rods = 30
        lens = rng.integers(2, 9, n_rods)
        off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
        nv = int(off[-1])
        x4 = np.zeros((nv, 4), np.float32)
        for r in range(n_rods):
            n = lens[r]
            start = rng.uniform(-0.3, 0.3, 3)
            d = rng.normal(size=3); d /= np.linalg.norm(d)
            x4[off[r]:off[r + 1], :3] = start + np.arange(n)[:, None] * 0.05 * d
        x4[:, 3] = rng.uniform(0.5, 1.5, nv)
        rbar = rng.uniform(0.005, 0.04, nv).astype(np.float32)
        group = rng.integers(0, 10 if trial % 2 else n_rods, n_rods).astype(np.int32)
        g = oracle.broadphase_f32(off, group, x4, rbar, brute=False)
        b = oracle.broadphase_f32(off, group, x4, rbar, brute=True)
        assert g.shape[0] > 10
        np.testing.assert_array_equal(g, b)


def test_broadphase_brute_force_is_the_fp32_predicate():
    """Every emitted pair passes, and every rejected pair fails, the FP32
    bounding-sphere test recomputed here with numpy float32 in the same order."""
    rng = np.random.default_rng(14)
    off = np.array([0, 3, 6, 9, 12], np.int32)
    x4 = np.zeros((12, 4), np.float32)
    x4[:, :3] = rng.uniform(-0.1, 0.1, (12, 3)).astype(np.float32)
    x4[:, 3] = 1.0
    rbar = np.full(12, 0.02, np.float32)
    group = np.arange(4, dtype=np.int32)
    pairs = {tuple(p) for p in oracle.broadphase_f32(off, group, x4, rbar, brute=True)}
    f = np.float32
    segs = [(r, v) for r in range(4) for v in range(off[r], off[r + 1] - 1)]
    sph = []
    for r, v in segs:
        x1, x2 = x4[v], x4[v + 1]
        c = (x1[:3] + x2[:3]) * f(0.5)
        d = x2[:3] - x1[:3]
        l2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
        R = f(0.5) * np.sqrt(f(l2)) + max(x1[3] * rbar[v], x2[3] * rbar[v + 1])
        sph.append((c, f(R), r))
    for a in range(len(segs)):
        for b in range(a + 1, len(segs)):
            ca, Ra, ra = sph[a]
            cb, Rb, rb = sph[b]
            e = ca - cb
            d2 = (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2]
            hit = (ra != rb) and d2 <= (Ra + Rb) * (Ra + Rb)
            assert hit == ((a, b) in pairs)


# --------------------------------------------------------------------------
# skinning (Sec. 7.4)
# --------------------------------------------------------------------------

def test_lbs_identity_and_rigid_motion():
    sc = S.muscle_rig(n_rods=5, mesh_verts=500)
    o = oracle.OracleScene(sc)
    out = o.skin()
    np.testing.assert_allclose(out, sc.mesh.rest, atol=1e-12)
    rng = np.random.default_rng(15)
    qR = _rand_quat(rng)
    R = np.stack([_rot(qR, e) for e in np.eye(3)], axis=1)
    t = np.array([1.0, 2.0, 3.0])
    st = o.get_state()
    o.set_state(x=_rigid(R, t, st["x"]), q=S.quat_mul(np.tile(qR, (sc.ns, 1)), st["q"]))
    np.testing.assert_allclose(o.skin(), _rigid(R, t, sc.mesh.rest), atol=1e-12)
    # uniform scale s about each frame centre scales the mesh about the
    # blended centre when all four frames of a vertex coincide
    o.set_state(x=st["x"], q=st["q"], s=np.full(sc.nv, 1.5))
    single = dataclasses.replace(sc.mesh, idx=np.repeat(sc.mesh.idx[:, :1], 4, axis=1))
    out = o.skin(single)
    seg_off = sc.rod_offsets - np.arange(sc.n_rods + 1)
    g = single.idx[:, 0]
    v0 = g + np.searchsorted(seg_off, g, side="right") - 1
    cm = 0.5 * (sc.rest_pos[v0] + sc.rest_pos[v0 + 1])
    np.testing.assert_allclose(out, cm + 1.5 * (sc.mesh.rest - cm), atol=1e-12)


# --------------------------------------------------------------------------
# colouring
# --------------------------------------------------------------------------

def test_colouring_separates_shared_dofs():
    sc = S.batching(n_rods=50)
    o = oracle.OracleScene(sc)
    segc, vtxc = o.colouring()
    off = sc.rod_offsets
    for r in range(sc.n_rods):
        v0, v1 = off[r], off[r + 1]
        s0 = v0 - r
        segs = segc[s0:s0 + (v1 - v0 - 1)]
        # adjacent segments share a vertex -> different colours
        assert (segs[1:] != segs[:-1]).all()
        vt = vtxc[v0:v1]
        assert vt[0] == -1 and vt[-1] == -1
        inner = vt[1:-1]
        # adjacent interior vertices share a segment rotation -> different colours
        assert (inner[1:] != inner[:-1]).all()
        assert set(np.unique(inner)).issubset({2, 3})


# --------------------------------------------------------------------------
# Surface bending (Sec. 5, E_bending; discrete Laplacian of Sec. 7.5)
# --------------------------------------------------------------------------

def test_surface_bending_laplacian_is_exact_for_quadratic_profiles():
    """The discrete scale Laplacian at a vertex with unequal neighbouring
    segments equals the second derivative of any quadratic profile."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        la, lb = rng.uniform(0.002, 0.05, 2)
        a, b, c = rng.normal(size=3)
        prof = lambda z: a + b * z + c * z * z
        C, _ = oracle.laplacian_constraint(prof(-la), prof(0.0), prof(lb), la, lb)
        np.testing.assert_allclose(C, 2 * c, rtol=1e-8, atol=1e-8)
        # a linear profile has no curvature
        C0, _ = oracle.laplacian_constraint(a - b * la, a, a + b * lb, la, lb)
        assert abs(C0) < 1e-9 * (1 + abs(b) / min(la, lb))


def test_surface_bending_jacobian_matches_finite_differences():
    rng = np.random.default_rng(8)
    for _ in range(10):
        la, lb = rng.uniform(0.005, 0.03, 2)
        s = rng.uniform(0.7, 1.3, 3)
        _, J = oracle.laplacian_constraint(*s, la, lb)
        eps = 1e-6
        for k in range(3):
            sp, sm = s.copy(), s.copy()
            sp[k] += eps
            sm[k] -= eps
            fd = (oracle.laplacian_constraint(*sp, la, lb)[0] - oracle.laplacian_constraint(*sm, la, lb)[0]) / (2 * eps)
            np.testing.assert_allclose(J[k], fd, rtol=1e-6)


def test_surface_bending_compliance_equals_integrated_energy_coefficient():
    """K per unit length equals the disc integral of the bending-approximation
    integrand ||R^T lap(phi) - Rbar^T lap(phibar)||_Kb^2 of Sec. 5 for a unit
    scale Laplacian: (k_x x^2 + k_y y^2) over the disc, k_x = k_y = 1/c_b."""
    r, l, cb = 0.03, 0.01, 2e-6
    sc = dataclasses.replace(_one_rod_scene(r=r, lbar=l, cb=cb), surface_bending=True)
    o = oracle.OracleScene(sc)
    X, Y, W = _disc_quadrature(r)
    kb = 1 / cb
    K_L = (kb * (X ** 2 + Y ** 2) * W).sum()
    np.testing.assert_allclose(1 / (o.laplacian_compliance(1) * l), K_L, rtol=1e-10)
    assert o.laplacian_compliance(0) == 0.0 and o.laplacian_compliance(sc.nv - 1) == 0.0


def _scale_bump_rod(surface):
    # soft first-order scale terms (X, G use the stretch compliance), stiff bending
    sc = _one_rod_scene(n=12, r=0.02, lbar=0.01, cs=1e-2, cb=1e-9, cv=1e-2)
    sc = dataclasses.replace(sc, surface_bending=surface, substeps=4, iterations=8, volume=False)
    o = oracle.OracleScene(sc)
    s = np.ones(sc.nv)
    s[6] = 1.3  # a sharp bump in the middle of a straight rod
    o.set_state(s=s)
    return sc, o


def _laplacian_residual(s, lb):
    out = []
    for i in range(1, len(s) - 1):
        out.append(oracle.laplacian_constraint(s[i - 1], s[i], s[i + 1], lb[i - 1], lb[i])[0])
    return np.sqrt(np.mean(np.square(out)))


def test_surface_bending_smooths_a_scale_bump():
    """With the constraint on, the scale profile's Laplacian falls faster than
    with the first-order terms (cross-section, scale gradient) alone; it acts on
    scales only, so positions and frames of the straight rod stay put."""
    res = {}
    for surface in (False, True):
        sc, o = _scale_bump_rod(surface)
        o.step(sc.dt, sc.substeps, sc.iterations)
        st = o.get_state()
        lb, _ = o.rest()
        res[surface] = _laplacian_residual(st["s"], lb)
        np.testing.assert_allclose(st["x"], sc.rest_pos, atol=1e-9)
    assert res[True] < 0.5 * res[False], res


# --------------------------------------------------------------------------
# Jacobi with averaging (Sec. 7 engine) as an alternative ordering
# --------------------------------------------------------------------------

def test_jacobi_first_vertex_equals_gauss_seidel_after_one_iteration():
    """With volume and surface bending off, a free rod's first vertex is moved
    only by the stretch/shear constraint of segment 0.  Gauss-Seidel projects
    that constraint first, on the predicted state, and nothing after it in the
    sweep touches the vertex; Jacobi projects it on the same state and divides
    by a count of one: after one iteration the vertex agrees exactly."""
    rng = np.random.default_rng(21)
    base = dataclasses.replace(_helix_scene(n_rods=3), volume=False)
    init_x = base.rest_pos + rng.normal(size=base.rest_pos.shape) * 2e-3
    init_q = S.quat_mul(S.axis_angle_quat(rng.normal(size=(base.ns, 3)) * 0.2), base.rest_quat)
    out = []
    for jacobi in (False, True):
        o = oracle.OracleScene(dataclasses.replace(base, jacobi=jacobi))
        o.set_state(x=init_x, q=init_q)
        assert o.step(dt=1 / 60, substeps=1, iterations=1) == 0
        out.append(o.get_state()["x"])
    first = base.rod_offsets[:-1]
    np.testing.assert_allclose(out[1][first], out[0][first], rtol=0, atol=1e-14)
    # elsewhere the two orderings differ
    assert np.abs(out[1] - out[0]).max() > 1e-6


def test_jacobi_converges_more_slowly_than_colouring():
    """E9-style: bars pulled to 2x instantly.  Each ordering approaches its own
    limit (Jacobi with averaging and full multiplier updates does not share
    Gauss-Seidel's fixed point), the distance falling with the iteration count;
    Gauss-Seidel, which carries a correction along the chain within one sweep,
    is closer to its limit at every count (the paper reports linear
    convergence for its Jacobi engine)."""
    n = 12
    sc = _one_rod_scene(n=n, r=0.01, lbar=0.01, cs=1e-9, cb=1e-7, cv=1e-9)
    sc = dataclasses.replace(sc, pin_vertex=np.array([0, n - 1], np.int32), pin_bone=np.array([-1, -1], np.int32),
                             pin_offset=np.array([[0, 0, 0], [2.0 * 0.01 * (n - 1), 0, 0]]))

    def run(jacobi, iters):
        o = oracle.OracleScene(dataclasses.replace(sc, jacobi=jacobi))
        assert o.step(dt=1 / 60, substeps=1, iterations=iters) == 0
        return o.get_state()["x"]

    dist = {}
    for jacobi, limit_iters in ((False, 4096), (True, 16384)):
        limit = run(jacobi, limit_iters)
        dist[jacobi] = [np.abs(run(jacobi, it) - limit).max() for it in (1, 4, 16, 64, 256)]
        d = dist[jacobi]
        assert all(a > b for a, b in zip(d, d[1:])), (jacobi, d)
    assert all(g < j for g, j in zip(dist[False][1:], dist[True][1:])), dist


# --------------------------------------------------------------------------
# Scale-invariant shape matching of bundles (Sec. 7.3)
# --------------------------------------------------------------------------

def test_polar_rotation_matches_svd():
    """Horn's quaternion eigenvector against numpy's SVD polar factor U diag(1,1,det) V^T."""
    rng = np.random.default_rng(31)
    for _ in range(50):
        A = rng.normal(size=(3, 3)) * rng.uniform(0.01, 10)
        U, _, Vt = np.linalg.svd(A)
        D = np.diag([1.0, 1.0, np.sign(np.linalg.det(U @ Vt))])
        np.testing.assert_allclose(oracle.polar_rotation(A), U @ D @ Vt, atol=1e-12)


def _free_bundle_scene():
    sc = S.bundled_muscles(n_muscles=3, fibers=7, n_verts=9, n_bones=3)
    return dataclasses.replace(sc, pin_vertex=np.zeros(0, np.int32), pin_bone=np.zeros(0, np.int32),
                               pin_offset=np.zeros((0, 3)), gravity=np.zeros(3), contacts=False)


def test_shape_match_keeps_an_exact_similarity_fixed():
    """A state that is a similarity s R (.) + t of the rest pose (positions,
    scales s, frames R q_bar) is a fixed point of the post-process."""
    rng = np.random.default_rng(32)
    sc = _free_bundle_scene()
    qR = _rand_quat(rng)
    R = np.stack([_rot(qR, e) for e in np.eye(3)], axis=1)
    s, t = 1.17, np.array([0.3, -0.2, 0.5])
    o = oracle.OracleScene(sc)
    x = sc.rest_pos @ R.T * s + t
    q = S.quat_mul(np.tile(qR, (sc.ns, 1)), sc.rest_quat)
    o.set_state(x=x, s=np.full(sc.nv, s), q=q)
    o.shape_match()
    st = o.get_state()
    np.testing.assert_allclose(st["x"], x, atol=1e-12)
    np.testing.assert_allclose(st["s"], s, atol=1e-12)
    np.testing.assert_allclose(np.abs((st["q"] * q).sum(1)), 1.0, atol=1e-12)


def test_shape_match_projects_onto_similarities_and_is_idempotent():
    """After the post-process every cross-section is an exact similarity of its
    rest (all pairwise distances scaled by one factor, equal scales), and a
    second application changes nothing."""
    rng = np.random.default_rng(33)
    sc = _free_bundle_scene()
    o = oracle.OracleScene(sc)
    x = sc.rest_pos + rng.normal(size=sc.rest_pos.shape) * 3e-3
    q = S.quat_mul(S.axis_angle_quat(rng.normal(size=(sc.ns, 3)) * 0.1), sc.rest_quat)
    o.set_state(x=x, s=rng.uniform(0.9, 1.1, sc.nv), q=q)
    o.shape_match()
    a = o.get_state()
    n_v = int(sc.rod_offsets[1] - sc.rod_offsets[0])
    for b in range(len(sc.bundle_offsets) - 1):
        rods = sc.bundle_rods[sc.bundle_offsets[b]:sc.bundle_offsets[b + 1]]
        for k in range(n_v):
            v = sc.rod_offsets[rods] + k
            d = np.linalg.norm(a["x"][v][:, None] - a["x"][v][None], axis=2)
            d0 = np.linalg.norm(sc.rest_pos[v][:, None] - sc.rest_pos[v][None], axis=2)
            ratio = d[d0 > 0] / d0[d0 > 0]
            np.testing.assert_allclose(ratio, ratio.mean(), rtol=1e-10)
            np.testing.assert_allclose(a["s"][v], a["s"][v][0], rtol=1e-12)
            np.testing.assert_allclose(ratio.mean(), a["s"][v][0], rtol=1e-10)
    o.shape_match()
    b2 = o.get_state()
    np.testing.assert_allclose(b2["x"], a["x"], atol=1e-12)
    np.testing.assert_allclose(b2["s"], a["s"], atol=1e-12)


def test_shape_match_minimises_the_bundle_energy():
    """Sec. 7.3's energy sum_i |T* T_bar_i - T_i|^2 with T_i = [s_i R_i, c_i]:
    the post-process's T* (read back from the projected state) scores no worse
    than nearby similarities."""
    rng = np.random.default_rng(34)
    sc = _free_bundle_scene()
    o = oracle.OracleScene(sc)
    x = sc.rest_pos + rng.normal(size=sc.rest_pos.shape) * 3e-3
    q = S.quat_mul(S.axis_angle_quat(rng.normal(size=(sc.ns, 3)) * 0.1), sc.rest_quat)
    sv = rng.uniform(0.9, 1.1, sc.nv)
    o.set_state(x=x, s=sv, q=q)
    o.shape_match()
    a = o.get_state()
    rods = sc.bundle_rods[:7]
    k = 3
    v = sc.rod_offsets[rods] + k
    g = sc.rod_offsets[rods] - rods + k

    def mats(qs):
        return np.stack([np.stack([_rot(qq, e) for e in np.eye(3)], axis=1) for qq in qs])

    Ri, Rb = mats(q[g]), mats(sc.rest_quat[g])
    Ti = [np.hstack([sv[vi] * Ri[j], x[vi][:, None]]) for j, vi in enumerate(v)]
    Tb = [np.vstack([np.hstack([Rb[j], sc.rest_pos[vi][:, None]]), [0, 0, 0, 1]]) for j, vi in enumerate(v)]

    def energy(s, R, c):
        Ts = np.vstack([np.hstack([s * R, c[:, None]]), [0, 0, 0, 1]])
        return sum(np.sum(((Ts @ Tb[j])[:3] - Ti[j]) ** 2) for j in range(len(v)))

    # T* from the projected state: c_i = s* R* c_bar_i + c*, frames R* R_bar
    s_star = a["s"][v][0]
    Rs = mats(a["q"][g])[0] @ Rb[0].T
    c_star = a["x"][v][0] - s_star * Rs @ sc.rest_pos[v][0]
    e0 = energy(s_star, Rs, c_star)
    for _ in range(50):
        dq = S.axis_angle_quat(rng.normal(size=3) * 1e-3)
        dR = np.stack([_rot(dq, e) for e in np.eye(3)], axis=1)
        e1 = energy(s_star * (1 + rng.normal() * 1e-3), dR @ Rs, c_star + rng.normal(size=3) * 1e-4)
        assert e1 >= e0 - 1e-12


def test_bundle_cross_sections_are_similarities_after_each_step():
    """Stepping pinned, animated muscles: every unpinned cross-section ends the
    substep as a similarity of its rest arrangement (the post-process runs
    after the iterations), while rods stay pinned to the bones."""
    sc = S.bundled_muscles(n_muscles=4, fibers=7, n_verts=10, n_bones=4)
    o = oracle.OracleScene(sc)
    for f in range(2):
        o.set_bones(*sc.bone_pose((f + 1) * sc.dt))
        assert o.step() == 0
    st = o.get_state()
    n_v = 10
    for b in range(len(sc.bundle_offsets) - 1):
        rods = sc.bundle_rods[sc.bundle_offsets[b]:sc.bundle_offsets[b + 1]]
        for k in range(1, n_v - 1):
            v = sc.rod_offsets[rods] + k
            d = np.linalg.norm(st["x"][v][:, None] - st["x"][v][None], axis=2)
            d0 = np.linalg.norm(sc.rest_pos[v][:, None] - sc.rest_pos[v][None], axis=2)
            ratio = d[d0 > 0] / d0[d0 > 0]
            np.testing.assert_allclose(ratio, ratio.mean(), rtol=1e-9)
            np.testing.assert_allclose(st["s"][v], st["s"][v][0], rtol=1e-9)


# --------------------------------------------------------------------------
# Muscle activation and the bone-driven warm start (Sec. 8.2)
# --------------------------------------------------------------------------

def test_zero_activation_is_the_rest_state():
    sc = S.muscle_rig(n_rods=6, mesh_verts=0)
    a, b = oracle.OracleScene(sc), oracle.OracleScene(sc)
    b.set_activation(np.zeros(sc.n_rods))
    for f in range(2):
        for o in (a, b):
            o.set_bones(*sc.bone_pose((f + 1) * sc.dt))
            assert o.step() == 0
    np.testing.assert_array_equal(a.get_state()["x"], b.get_state()["x"])
    with pytest.raises(ValueError):
        b.set_activation(np.full(sc.n_rods, 0.95))


def test_activation_keeps_mass_and_rest_volume():
    sc = _one_rod_scene(n=10, r=0.02, lbar=0.01)
    o = oracle.OracleScene(sc)
    m0 = [o.vertex_inverse_inertia(i)[0] for i in range(sc.nv)]
    lb0, _ = o.rest()
    o.set_activation(np.array([0.4]))
    m1 = [o.vertex_inverse_inertia(i)[0] for i in range(sc.nv)]
    lb1, _ = o.rest()
    np.testing.assert_allclose(m1, m0, rtol=1e-12)
    np.testing.assert_allclose(lb1, 0.6 * lb0, rtol=1e-12)


def test_activated_free_rod_shortens_and_bulges():
    """A free, straight rod (no pins, no gravity) with activation a relaxes to
    (1 - a) of its length and 1/sqrt(1 - a) of its radius: fibre shortening
    bulges the muscle at constant volume."""
    a = 0.3
    sc = dataclasses.replace(_one_rod_scene(n=10, r=0.01, lbar=0.01, cs=1e-8, cb=1e-6, cv=1e-8),
                             substeps=10, iterations=8)
    o = oracle.OracleScene(sc)
    o.set_activation(np.array([a]))
    for _ in range(40):
        assert o.step() == 0
    st = o.get_state()
    length = np.linalg.norm(np.diff(st["x"], axis=0), axis=1).sum()
    L0 = 0.01 * (sc.nv - 1)
    np.testing.assert_allclose(length, (1 - a) * L0, rtol=2e-2)
    radius = st["s"] * sc.radius / math.sqrt(1 - a)
    np.testing.assert_allclose(radius[1:-1], sc.radius[1:-1] / math.sqrt(1 - a), rtol=2e-2)


def _translating_bones_scene(d0, d1, warm):
    """One rod pinned at both ends to two bones; the bones translate by d0, d1."""
    sc = dataclasses.replace(S.muscle_rig(n_rods=1, n_bones=2, mesh_verts=0), warm_start=warm,
                             gravity=np.zeros(3))
    q0, t0 = sc.bones.pose(0.0)
    return sc, q0, t0, t0 + np.stack([d0, d1])


def test_warm_start_blends_the_two_bone_motions_by_arclength():
    """Bones translating by d0 and d1: before any solving (one substep, no
    iterations, zero velocity and gravity) every vertex moves by
    (1 - t) d0 + t d1, t its arclength fraction; without the warm start only
    the pinned ends move."""
    d0, d1 = np.array([0.05, 0.0, 0.01]), np.array([-0.02, 0.03, 0.0])
    for warm in (True, False):
        sc, q0, t0, t1 = _translating_bones_scene(d0, d1, warm)
        o = oracle.OracleScene(sc)
        o.set_bones(q0, t1)
        assert o.step(dt=1 / 60, substeps=1, iterations=0) == 0
        x = o.get_state()["x"]
        seg = np.linalg.norm(np.diff(sc.rest_pos, axis=0), axis=1)
        t = np.concatenate([[0.0], np.cumsum(seg)]) / seg.sum()
        expect = sc.rest_pos + (1 - t)[:, None] * d0 + t[:, None] * d1 if warm else sc.rest_pos.copy()
        if not warm:
            expect[0] += d0
            expect[-1] += d1
        np.testing.assert_allclose(x, expect, atol=1e-12)


def test_warm_start_lowers_the_residual_of_fast_bone_motion():
    """Sec. 8.2: initialising from the bones speeds up convergence in fast
    motion -- after a frame in which the bones jump, the constraint residual is
    smaller with the warm start."""
    res = {}
    for warm in (False, True):
        sc, q0, t0, t1 = _translating_bones_scene(np.array([0.08, 0.02, 0.0]), np.array([0.05, -0.04, 0.03]), warm)
        o = oracle.OracleScene(sc)
        o.set_bones(q0, t1)
        assert o.step(dt=1 / 60, substeps=2, iterations=2) == 0
        res[warm] = o.constraint_rms()["S"]
    assert res[True] < 0.5 * res[False], res


@pytest.mark.parametrize("name", ["hair", "muscle_rig"])
def test_oracle_threads_give_identical_results(name):
    """The OpenMP colour sweeps and contact pass (pairs in parallel, sums in
    pair order) give bitwise the single-thread result."""
    # hair: 400 strands on a 3 cm sphere (about 8k pairs), reaching the floor plane by frame 3
    sc = S.hair(n_rods=400, sphere=0.03, box=0.12) if name == "hair" else S.muscle_rig(mesh_verts=0)
    out = []
    for threads in (1, 3):
        o = oracle.OracleScene(sc, threads=threads)
        for _ in range(4):
            assert o.frame() == 0
        assert len(o.last_pairs()) > 0
        out.append(o.get_state())
    for k in out[0]:
        np.testing.assert_array_equal(out[0][k], out[1][k])
