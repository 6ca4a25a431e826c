"""Pins of the FP64 oracle against facts other than itself.

Each test checks the oracle against a closed form, an invariant, a textbook
special case or brute force, chosen so that a plausible mistake (a dropped
term, a wrong sign or index, a transposed operand, a different ordering of
Algorithm 1) fails at least one of them.  CPU only.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2106_13281_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers
def qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def axis_angle(axis, ang):
    axis = np.asarray(axis, dtype=np.float64) / np.linalg.norm(axis)
    return np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * axis])


def single_body(mass=2.0, inertia=(0.3, 0.5, 0.7), g=(0, 0, 0), dt=0.05, substeps=10):
    sb = S.SceneBuilder(dt=dt, substeps=substeps, gravity=g)
    sb.body("b", mass, inertia, (0, 0, 0))
    return sb.build()


def state_of(desc, pos=None, quat=None, vel=None, ang=None, n=1):
    B = len(desc["mass"])
    st = np.zeros((n, B, 13))
    st[:, :, 3] = 1.0
    st[:, :, 0:3] = desc["rest_pos"]
    st[:, :, 3:7] = desc["rest_rot"]
    for k, v in ((0, pos), (3, quat), (7, vel), (10, ang)):
        if v is not None:
            st[:, 0, k:k + len(v)] = v
    return st


def rotmats(q):
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                  2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                  2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)
    return R.reshape(q.shape[:-1] + (3, 3))


def anchor_errors(desc, st):
    R = rotmats(st[..., 3:7])
    out = []
    for j in range(len(desc["parent"])):
        p, c = desc["parent"][j], desc["child"][j]
        pp = st[..., p, :3] + np.einsum("...ij,j->...i", R[..., p, :, :], desc["parent_offset"][j])
        pc = st[..., c, :3] + np.einsum("...ij,j->...i", R[..., c, :, :], desc["child_offset"][j])
        out.append(np.linalg.norm(pp - pc, axis=-1))
    return np.stack(out, -1)


def no_contacts(desc):
    d = dict(desc)
    d["pair_a"] = np.zeros(0, dtype=np.int32)
    d["pair_b"] = np.zeros(0, dtype=np.int32)
    return d


# ----------------------------------------------------------------- integrators
def test_free_fall_closed_form():
    """x_n = x0 + n h v0 + g h^2 n(n-1)/2 and v_n = v0 + n h g (Algorithm 1:
    kinematic first, then the potential update)."""
    g = (0.3, -0.2, -9.81)
    d = single_body(g=g)
    x0, v0 = np.array([0.1, -0.4, 2.0]), np.array([1.5, 0.25, 3.0])
    st = state_of(d, pos=x0, vel=v0)
    T = 7
    out = orc.rollout(d, st, np.zeros((T, 1, 0)))
    n, h = T * 10, 0.005
    assert np.allclose(out[0, 0, 7:10], v0 + n * h * np.array(g), atol=1e-12, rtol=0)
    assert np.allclose(out[0, 0, 0:3], x0 + n * h * v0 + np.array(g) * h * h * n * (n - 1) / 2, atol=1e-12, rtol=0)


def test_free_spin_closed_form():
    """Torque-free: w constant; q_n = Rot(w_hat, 2 n atan(h|w|/2)) q0 (world-frame update)."""
    d = single_body(inertia=(0.2, 0.9, 1.7))
    rng = np.random.default_rng(0)
    w = rng.normal(size=3) * 3.0
    q0 = axis_angle(rng.normal(size=3), 1.1)
    st = state_of(d, quat=q0, ang=w)
    T = 5
    out = orc.rollout(d, st, np.zeros((T, 1, 0)))
    n, h = T * 10, 0.005
    ang = 2 * n * math.atan(h * np.linalg.norm(w) / 2)
    expect = qmul(axis_angle(w, ang), q0)
    assert np.allclose(out[0, 0, 10:13], w, atol=1e-13)
    assert np.allclose(out[0, 0, 3:7], expect, atol=1e-12)
    assert abs(np.linalg.norm(out[0, 0, 3:7]) - 1) < 1e-13


def hinge_system(gear=2.0, ca=0.5, I=0.8, lim=(-180, 180), kl=50.0, g=(0, 0, 0), dt=0.01, substeps=1, off=0.0,
                 ka=40.0, c=5.0):
    sb = S.SceneBuilder(dt=dt, substeps=substeps, gravity=g)
    p = sb.body("P", 1.0, (1, 1, 1), (0, 0, 0), frozen_pos=(1, 1, 1), frozen_rot=(1, 1, 1))
    cb = sb.body("C", 1.0, (I, I, I), (0, 0, -off))
    j = sb.joint(p, cb, anchor=(0, 0, 0), axis=(1, 0, 0), ref=(0, 1, 0), stiffness=10000.0, spring_damping=c,
                 angular_stiffness=ka, angular_damping=ca, limits=(lim,), limit_stiffness=kl)
    sb.actuator(j, 0, gear)
    return sb.build()


def test_damped_hinge_closed_form():
    """Frozen parent, child COM on the hinge axis at the anchor, no gravity,
    constant torque: w_n = w_inf + (w0 - w_inf) rho^n with rho = 1 - h c_a/I,
    w_inf = tau/c_a; angle_n = sum of 2 atan(h w_i / 2)."""
    gear, ca, I, a = 2.0, 0.5, 0.8, 0.6
    d = hinge_system(gear=gear, ca=ca, I=I)
    st = orc.default_qp(d, 1)
    w0 = 0.7
    st[0, 1, 10:13] = [w0, 0, 0]
    T = 400
    out, tr = orc.rollout(d, st, np.full((T, 1, 1), a), traj=True)
    h = 0.01
    tau = gear * a
    w_inf = tau / ca
    rho = 1 - h * ca / I
    n = np.arange(1, T + 1)
    w_expect = w_inf + (w0 - w_inf) * rho ** n
    assert np.allclose(tr[:, 0, 1, 10], w_expect, atol=1e-11, rtol=0)
    w_prev = np.concatenate([[w0], w_expect[:-1]])
    theta = np.cumsum(2 * np.arctan(h * w_prev / 2))
    ang = np.array([orc.joint_angles(d, tr[t])[0, 0] for t in range(T)])
    wrapped = np.angle(np.exp(1j * theta))
    assert np.allclose(ang, wrapped, atol=1e-10)
    # the anchors stay together and the hinge axes stay aligned
    assert anchor_errors(d, tr).max() < 1e-12


def test_hinge_limit_static_balance():
    """Constant torque into the upper limit: at rest k_l (theta - hi) = tau."""
    gear, kl = 10.0, 100.0
    d = hinge_system(gear=gear, ca=1.0, I=1.0, lim=(-30, 30), kl=kl)
    st = orc.default_qp(d, 1)
    out = orc.rollout(d, st, np.full((4000, 1, 1), 1.0))
    theta = orc.joint_angles(d, out)[0, 0]
    assert abs(theta - (math.radians(30) + gear / kl)) < 1e-9
    out2 = orc.rollout(d, st, np.full((4000, 1, 1), -1.0))
    assert abs(orc.joint_angles(d, out2)[0, 0] - (math.radians(-30) - gear / kl)) < 1e-9


def test_appendix_a_system_and_equilibrium():
    """The App. A system matches the golden spec; hanging at rest its spring
    stretches by m g / k (the steady state of the step)."""
    gold = json.load(open(os.path.join(GOLDEN, "appendix_a.json")))
    d = S.appendix_a()
    assert d["substeps"] == gold["substeps"] and d["dt"] == gold["dt"]
    assert np.allclose(d["gravity"], gold["gravity"])
    for b, gb in enumerate(gold["bodies"]):
        assert d["mass"][b] == gb["mass"] and np.allclose(d["inertia"][b], gb["inertia"])
        assert list(d["frozen_pos"][b]) == gb["frozen_pos"] and list(d["frozen_rot"][b]) == gb["frozen_rot"]
    assert d["stiffness"][0] == gold["joint"]["stiffness"]
    assert np.allclose(d["child_offset"][0], gold["joint"]["child_offset"])
    assert np.allclose([d["limit_lo"][0][0], d["limit_hi"][0][0]], gold["joint"]["angle_limit_deg"])
    st = orc.default_qp(d, 1)
    out = orc.rollout(d, st, np.zeros((3000, 1, 0)))
    gap = anchor_errors(d, out)[0, 0]
    assert abs(gap - 1.0 * 9.8 / 10000.0) < 1e-9
    assert np.allclose(out[0, 0], st[0, 0])  # the frozen parent never moves


def test_quaternion_norm_preserved():
    d = S.quadruped()
    rp, rr, ang = S.initial_conditions(d, 4, 0)
    st = orc.default_qp(d, 4, rp, rr, ang)
    a = S.actions(d, 4, 20, 0)
    out = orc.rollout(d, st, a)
    assert np.abs(np.linalg.norm(out[..., 3:7], axis=-1) - 1).max() < 1e-13


# ----------------------------------------------------------------- contacts
def sphere_scene(inertia=None, r=0.2, m=1.5, length=None, axis=(0, 0, 1), friction=1.0, baumgarte=0.1):
    sb = S.SceneBuilder(dt=0.05, substeps=10, gravity=(0, 0, -9.81), baumgarte=baumgarte)
    L = 2 * r if length is None else length
    b = sb.capsule_body("s", m, r, L, (0, 0, 1.0), axis, friction=friction, inertia=inertia)
    g = sb.plane(friction=1.0)
    sb.pair(sb.collider_of(b), g)
    return sb.build()


def test_resting_sphere_height():
    """Steady penetration d* = g h^2 / beta under Algorithm 1 (contacts see
    the velocities before the potential update)."""
    r, h, g, beta = 0.2, 0.005, 9.81, 0.1
    d = sphere_scene(r=r)
    st = state_of(d, pos=[0, 0, r])
    out = orc.rollout(d, st, np.zeros((400, 1, 0)))
    assert abs(out[0, 0, 2] - (r - g * h * h / beta)) < 1e-12
    assert np.abs(out[0, 0, 7:13]).max() < 1e-12


def test_resting_capsule_heights():
    """Vertical capsule: one contact, same depth as the sphere.  Horizontal
    capsule: two contacts averaged, d* = g h^2 / (alpha beta) with
    alpha = (1/m) / (1/m + s^2 / I_t)."""
    r, L, m, h, g, beta = 0.1, 0.6, 2.0, 0.005, 9.81, 0.1
    s = L / 2 - r
    I = S.capsule_inertia(m, r, L)
    d = sphere_scene(r=r, length=L, m=m, inertia=I)
    st = state_of(d, pos=[0, 0, s + r])
    out = orc.rollout(d, st, np.zeros((400, 1, 0)))
    assert abs(out[0, 0, 2] - (s + r - g * h * h / beta)) < 1e-12
    dh = sphere_scene(r=r, length=L, m=m, inertia=I, axis=(1, 0, 0))
    st = state_of(dh, pos=[0, 0, r])
    out = orc.rollout(dh, st, np.zeros((400, 1, 0)))
    alpha = (1 / m) / (1 / m + s * s / I[0])
    assert abs(out[0, 0, 2] - (r - g * h * h / (alpha * beta))) < 1e-12


def test_resting_box_height():
    """Box on a plane: four corner contacts averaged, k_n = 1/m + hy^2/Ixx + hx^2/Iyy."""
    m, half, h, g, beta = 0.5, np.array([0.05, 0.08, 0.03]), 0.005, 9.81, 0.1
    sb = S.SceneBuilder(dt=0.05, substeps=10, gravity=(0, 0, -g))
    I = S.box_inertia(m, half)
    b = sb.body("box", m, I, (0, 0, 0))
    bc = sb.collider(b, S.BOX, half=half)
    sb.pair(bc, sb.plane())
    d = sb.build()
    st = state_of(d, pos=[0, 0, half[2]])
    out = orc.rollout(d, st, np.zeros((400, 1, 0)))
    kn = 1 / m + half[1] ** 2 / I[0] + half[0] ** 2 / I[1]
    alpha = (1 / m) / kn
    assert abs(out[0, 0, 2] - (half[2] - g * h * h / (alpha * beta))) < 1e-12


def test_sliding_sphere_friction():
    """Solid sphere (I = 2/5 m r^2) in converged contact given speed u0: while
    sliding the speed drops by mu g h per substep; rolling sets in at 5/7 u0
    (textbook), within O(h)."""
    r, m, g, h, u0 = 0.2, 1.5, 9.81, 0.005, 2.0
    I = 0.4 * m * r * r
    d = sphere_scene(r=r, m=m, inertia=(I, I, I))
    st = state_of(d, pos=[0, 0, r])
    st = orc.rollout(d, st, np.zeros((100, 1, 0)))  # settle the contact
    st[0, 0, 7:13] = [u0, 0, 0, 0, 0, 0]
    d1 = dict(d, substeps=1, dt=h)
    speeds = [u0]
    cur = st
    for _ in range(20):
        cur = orc.rollout(d1, cur, np.zeros((1, 1, 0)))
        speeds.append(cur[0, 0, 7])
    dec = -np.diff(speeds[2:12])
    assert np.allclose(dec, g * h, rtol=1e-6)
    fin = orc.rollout(d, st, np.zeros((200, 1, 0)))
    assert abs(fin[0, 0, 7] - 5.0 / 7.0 * u0) < 0.02 * u0
    # rolling without slipping at the end: contact point velocity v - w_y r = 0
    assert abs(fin[0, 0, 7] - fin[0, 0, 11] * r) < 1e-6


def test_segment_closest_brute_force():
    rng = np.random.default_rng(1)
    cases = []
    for _ in range(40):
        cases.append(rng.normal(size=(4, 3)))
    P = np.array([0.0, 0, 0])
    cases.append(np.array([P, [1, 0, 0], [0, 0.5, 0], [1, 0.5, 0]]))      # parallel
    cases.append(np.array([P, [1, 0, 0], [2, 0.5, 0], [3, 0.5, 0]]))      # collinear-ish, disjoint
    cases.append(np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0.3], [0, 1, 0.3]]))  # crossing
    cases.append(np.array([P, P, [0.3, 0.4, 0], [1, 2, 3]]))              # zero-length first
    cases.append(np.array([[0.2, 0.1, 0], [1, 0, 1], [0.5, 0.5, 0.5], [0.5, 0.5, 0.5]]))  # zero-length second
    grid = np.linspace(0, 1, 401)
    for P1, Q1, P2, Q2 in cases:
        s, t = orc.segment_closest(P1, Q1, P2, Q2)
        assert -1e-15 <= s <= 1 + 1e-15 and -1e-15 <= t <= 1 + 1e-15
        got = np.linalg.norm(P1 + s * (Q1 - P1) - P2 - t * (Q2 - P2))
        A = P1[None, None, :] + grid[:, None, None] * (Q1 - P1)
        Bp = P2[None, None, :] + grid[None, :, None] * (Q2 - P2)
        dd = np.linalg.norm(A - Bp, axis=-1)
        i, j = np.unravel_index(np.argmin(dd), dd.shape)
        # local refinement of the sampled minimum
        from scipy.optimize import minimize
        f = lambda x: np.linalg.norm(P1 + np.clip(x[0], 0, 1) * (Q1 - P1) - P2 - np.clip(x[1], 0, 1) * (Q2 - P2))
        best = min(dd[i, j], minimize(f, [grid[i], grid[j]], method="Nelder-Mead",
                                      options=dict(xatol=1e-12, fatol=1e-14, maxiter=4000)).fun)
        assert got <= best + 1e-9, (got, best)


def test_capsule_box_brute_force():
    rng = np.random.default_rng(2)
    tgrid = np.linspace(0, 1, 20001)
    n_hit = n_inside = 0
    for _ in range(120):
        he = rng.uniform(0.05, 0.3, size=3)
        c = rng.normal(size=3) * 0.2
        q = axis_angle(rng.normal(size=3), rng.uniform(0, 3))
        P = c + rng.normal(size=3) * 0.4
        Q = c + rng.normal(size=3) * 0.4
        r = rng.uniform(0.03, 0.2)
        R = rotmats(q)
        pts = P[None] + tgrid[:, None] * (Q - P)[None]
        loc = (pts - c) @ R
        res = loc - np.clip(loc, -he, he)
        dist = np.linalg.norm(res, axis=1)
        mind = dist.min()
        out = orc.capsule_box(P, Q, r, c, q, he)
        step = np.linalg.norm(Q - P) * (tgrid[1] - tgrid[0])  # sampling step along the segment
        pen = (he[None, :] - np.abs(loc)).min(axis=1)
        if pen.max() > 1e-3:  # the segment clearly meets the box: point closest to the box centre
            assert out is not None
            depth, n, p = out
            j = np.argmin(np.linalg.norm(loc, axis=1))
            gaps = np.sort(he - np.abs(loc[j]))
            assert abs(depth - (r + pen[j])) <= step + 1e-9
            if gaps[1] - gaps[0] > 4 * step:  # a unique face of least penetration
                k = np.argmin(he - np.abs(loc[j]))
                nl = np.zeros(3)
                nl[k] = np.sign(loc[j][k])
                assert np.allclose(n, R @ nl, atol=1e-12)
                p_ref = c + R @ (loc[j] + 0.5 * (pen[j] - r) * nl)
                assert np.linalg.norm(p - p_ref) <= 2 * step + 1e-9
            n_inside += 1
        if mind > 1e-6:
            if r - mind > 1e-9:
                assert out is not None
                depth, n, p = out
                # the exact minimum lies at or below the sampled one, by at most one sampling step
                assert -1e-12 <= depth - (r - mind) <= step + 1e-9
                n_hit += 1
            elif r - mind < -step - 1e-9:
                assert out is None
    assert n_hit > 5 and n_inside > 5


def test_closest_parameter_minimises_distance():
    """The segment parameter is the exact minimiser of the convex piecewise-
    quadratic segment-box squared distance: never above the best of a fine
    grid, and at the grid's minimiser where that minimiser is unique."""
    rng = np.random.default_rng(3)
    tgrid = np.linspace(0, 1, 100001)
    n_int = 0
    for _ in range(60):
        he = rng.uniform(0.05, 0.3, size=3)
        Pl = rng.normal(size=3) * 0.5
        dl = rng.normal(size=3) * 0.5
        t = orc.seg_box_param(Pl, dl, he)
        f = lambda tt: np.sum((Pl + np.outer(tt, dl) - np.clip(Pl + np.outer(tt, dl), -he, he)) ** 2, axis=-1)
        fg = f(tgrid)
        assert 0.0 <= t <= 1.0
        assert f(np.array([t]))[0] <= fg.min() + 1e-15
        if fg.min() > 1e-6:  # strictly convex near the minimiser: the parameter is unique
            assert abs(t - tgrid[np.argmin(fg)]) <= 2e-5
            n_int += 0.0 < t < 1.0
    he = np.array([0.1, 0.1, 0.1])
    # beyond the +x face, moving away from it: the start point
    assert orc.seg_box_param(np.array([0.2, 0.0, 0.3]), np.array([0.3, 0.0, 0.0]), he) == 0.0
    # e = (-0.5 + t, 0, 0.5 - 0.2 t): on t in [0.6, 1] the squared distance is
    # (t - 0.6)^2 + (0.4 - 0.2 t)^2, stationary at t = 1.36 / 2.08 = 17/26
    t = orc.seg_box_param(np.array([-0.5, 0.0, 0.5]), np.array([1.0, 0.0, -0.2]), he)
    assert abs(t - 17.0 / 26.0) < 1e-14
    # parallel to the top face, 0.2 above it: every t in [0.4, 0.6] is a minimiser
    t = orc.seg_box_param(np.array([-0.5, 0.0, 0.3]), np.array([1.0, 0.0, 0.0]), he)
    assert 0.4 - 1e-15 <= t <= 0.6 + 1e-15
    assert n_int > 5


def test_box_plane_depth_is_lowest_corner():
    sb = S.SceneBuilder()
    half = np.array([0.1, 0.2, 0.05])
    b = sb.body("box", 1.0, S.box_inertia(1.0, half), (0, 0, 0))
    bc = sb.collider(b, S.BOX, half=half)
    sb.pair(bc, sb.plane())
    d = sb.build()
    rng = np.random.default_rng(4)
    signs = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)])
    for _ in range(20):
        q = axis_angle(rng.normal(size=3), rng.uniform(0, 3))
        x = np.array([0.0, 0.0, rng.uniform(-0.1, 0.15)])
        st = state_of(d, pos=x, quat=q)[0]
        corners = x + (signs * half) @ rotmats(q).T
        cts = orc.contacts(d, st)
        below = corners[corners[:, 2] < 0]
        assert len(cts) == len(below)
        if len(below):
            assert abs(max(c[2] for c in cts) + corners[:, 2].min()) < 1e-12


# ----------------------------------------------------------------- invariants
def test_linear_momentum_exact_without_gravity_and_contacts():
    """Every joint and actuator term is equal and opposite: sum m v is constant
    to roundoff with g = 0, no contacts, random actions and damping on."""
    d = no_contacts(S.quadruped())
    d["gravity"] = np.zeros(3)
    rp, rr, ang = S.initial_conditions(d, 4, 5)
    st = orc.default_qp(d, 4, rp, rr, ang)
    st[:, :, 7:13] = np.random.default_rng(5).normal(size=st[:, :, 7:13].shape)
    a = S.actions(d, 4, 40, 5)
    _, m0 = orc.energy_momentum(d, st)
    out = orc.rollout(d, st, a)
    _, m1 = orc.energy_momentum(d, out)
    scale = np.abs(m0[:, :3]).max() + 1
    assert np.abs(m1[:, :3] - m0[:, :3]).max() < 1e-12 * scale * 1e3


def test_angular_momentum_exact_isotropic_no_linear_damping():
    """With isotropic inertia, no gravity, contacts or linear joint damping,
    the step conserves angular momentum to roundoff: spring forces act along
    the anchor separation and all torques come in equal and opposite pairs."""
    d = no_contacts(S.quadruped())
    d["gravity"] = np.zeros(3)
    d["spring_damping"] = np.zeros_like(d["spring_damping"])
    assert np.allclose(d["inertia"], 1.0)
    rp, rr, ang = S.initial_conditions(d, 4, 6)
    st = orc.default_qp(d, 4, rp, rr, ang)
    st[:, :, 7:13] = np.random.default_rng(6).normal(size=st[:, :, 7:13].shape)
    a = S.actions(d, 4, 40, 6)
    _, m0 = orc.energy_momentum(d, st)
    out = orc.rollout(d, st, a)
    _, m1 = orc.energy_momentum(d, out)
    assert np.abs(m1[:, 3:] - m0[:, 3:]).max() < 1e-9
    # linear damping breaks it (the damper force is not along the separation)
    d2 = dict(d, spring_damping=np.full_like(d["spring_damping"], 30.0))
    _, m2 = orc.energy_momentum(d2, orc.rollout(d2, st, a))
    assert np.abs(m2[:, 3:] - m0[:, 3:]).max() > 1e-6


def astronaut(h_substeps, damping=False):
    """The Sec. 6 conservation protocol: no damping, collisions or gravity."""
    d = no_contacts(S.biped())
    d["gravity"] = np.zeros(3)
    if not damping:
        d["spring_damping"] = np.zeros_like(d["spring_damping"])
        d["angular_damping"] = np.zeros_like(d["angular_damping"])
    d["substeps"] = h_substeps
    return d


def test_energy_drift_falls_with_step_size():
    """Actuators off, random 1 m/s kicks, 1 s of simulation: the energy drift
    shrinks as h shrinks (Sec. 6 energy protocol)."""
    rng = np.random.default_rng(7)
    drifts = []
    for subs in (10, 20, 40):
        d = astronaut(subs)
        rp, rr, ang = S.initial_conditions(d, 8, 7, angle_sigma=0.05)
        st = orc.default_qp(d, 8, rp, rr, ang)
        kick = rng.normal(size=(8, st.shape[1], 3))
        kick /= np.linalg.norm(kick, axis=-1, keepdims=True)
        st[:, :, 7:10] = kick
        rng = np.random.default_rng(7)
        e0, _ = orc.energy_momentum(d, st)
        out = orc.rollout(d, st, np.zeros((20, 8, len(d["gear"]))))
        e1, _ = orc.energy_momentum(d, out)
        drifts.append(np.mean(np.abs(e1 - e0) / e0))
    assert drifts[0] < 0.1  # 7.6% at h = 5 ms, 2.5% at 2.5 ms, 1.5% at 1.25 ms
    assert drifts[1] < drifts[0] and drifts[2] < drifts[1]


def test_astronaut_momentum_protocol():
    """Random ~0.5 N m actuation for 1 s with damping, collisions and gravity
    off: linear momentum exact; angular momentum exact for these isotropic
    bodies when the linear joint damper is off."""
    d = astronaut(10)
    d["gear"] = np.full_like(d["gear"], 0.5)
    rp, rr, ang = S.initial_conditions(d, 8, 8)
    st = orc.default_qp(d, 8, rp, rr, ang)
    a = S.actions(d, 8, 20, 8)
    _, m0 = orc.energy_momentum(d, st)
    out = orc.rollout(d, st, a)
    _, m1 = orc.energy_momentum(d, out)
    assert np.abs(m1 - m0).max() < 1e-10


# ----------------------------------------------------------------- default_qp / angles
@pytest.mark.parametrize("name", ["quadruped", "biped", "pendulum", "arm_box", "appendix_a"])
def test_default_qp_valid_configuration(name):
    """default_qp places every joint's anchors together and reproduces the
    requested joint angles (hinge angle and X-Y-Z Euler decomposition)."""
    d = S.SCENES[name]()
    rp, rr, ang = S.initial_conditions(d, 6, 9, height_jitter=0.05)
    st = orc.default_qp(d, 6, rp, rr, ang)
    if len(d["parent"]):
        assert anchor_errors(d, st).max() < 1e-12
        back = orc.joint_angles(d, st)
        assert np.allclose(back, ang, atol=1e-12)
    assert np.allclose(st[:, 0, 0:3], rp)
    assert np.abs(np.linalg.norm(st[..., 3:7], axis=-1) - 1).max() < 1e-14


def test_euler_round_trip_large_angles():
    d = S.biped()
    rng = np.random.default_rng(10)
    D = S.n_dof(d)
    ang = rng.uniform(-1.2, 1.2, size=(20, D))
    st = orc.default_qp(d, 20, None, None, ang)
    assert np.allclose(orc.joint_angles(d, st), ang, atol=1e-11)


# ----------------------------------------------------------------- adjoint
def small_quadruped_inputs(N=3, T=6, seed=11):
    d = S.quadruped()
    rp, rr, ang = S.initial_conditions(d, N, seed, height_jitter=0.05)
    st = orc.default_qp(d, N, rp, rr, ang)
    st[:, 0, 2] -= 0.38  # start with feet near the ground so contacts occur
    a = S.actions(d, N, T, seed).astype(np.float64)
    return d, st, a


def test_adjoint_dot_product():
    """<u, J v> (forward-mode duals) equals <J^T u, v> (reverse-mode tape)."""
    d, st, a = small_quadruped_inputs()
    rng = np.random.default_rng(12)
    u = rng.normal(size=st.shape)
    v_s, v_a = rng.normal(size=st.shape), rng.normal(size=a.shape)
    ds, _ = orc.jvp(d, st, a, v_s, v_a)
    ga, gs = orc.vjp(d, st, a, u)
    lhs = np.sum(u * ds)
    rhs = np.sum(ga * v_a) + np.sum(gs * v_s)
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))
    _, _, cc = orc.rollout(d, st, a, traj=True, contact_count=True)
    assert cc.sum() > 0  # contacts took part


def test_adjoint_vs_central_differences():
    """FP64 central differences (h = 1e-6) of a scalar loss match the tape
    gradient wherever the +h and -h runs take the same branches (contact
    activation, friction stick/slip, limits, clamps) as the unperturbed run."""
    d, st, a = small_quadruped_inputs(N=2, T=5)
    rng = np.random.default_rng(13)
    u = rng.normal(size=st.shape)

    def loss(s, act):
        out, sig = orc.rollout(d, s, act, branch_signature=True)
        return float(np.sum(u * out)), sig

    ga, gs = orc.vjp(d, st, a, u)
    _, sig0 = loss(st, a)
    eps = 1e-6
    checked = 0
    for _ in range(30):
        if rng.uniform() < 0.5:
            idx = tuple(rng.integers(0, n) for n in a.shape)
            ap, am = a.copy(), a.copy()
            ap[idx] += eps
            am[idx] -= eps
            (lp, s1), (lm, s2) = loss(st, ap), loss(st, am)
            g = ga[idx]
        else:
            n, b, k = rng.integers(0, st.shape[0]), rng.integers(0, st.shape[1]), rng.choice([0, 1, 2, 7, 8, 9, 10, 11, 12])
            sp, sm = st.copy(), st.copy()
            sp[n, b, k] += eps
            sm[n, b, k] -= eps
            (lp, s1), (lm, s2) = loss(sp, a), loss(sm, a)
            g = gs[n, b, k]
        if not (np.array_equal(s1, sig0) and np.array_equal(s2, sig0)):
            continue
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g) <= 1e-5 * max(1.0, abs(g)), (fd, g)
        checked += 1
    assert checked >= 20


def test_flop_counter_categories():
    d = S.quadruped()
    rp, rr, ang = S.initial_conditions(d, 2, 0)
    st = orc.default_qp(d, 2, rp, rr, ang)
    a = S.actions(d, 2, 3, 0)
    counts, na = orc.flops(d, st, a)
    for k in ("body", "joint", "actuator", "detect", "integrate"):
        assert counts[k] > 0
    # per-body work is per body and substep: 2 envs x 3 steps x 10 substeps x 9 bodies
    assert counts["body"] % (2 * 3 * 10 * 9) == 0


def test_reverse_op_count_is_additive():
    """The tape's reverse-op count (the reverse pass's algorithmic flops) adds
    over environments and steps: two identical environments count twice one,
    and a free body's steps (no contact, no joint) all cost the same."""
    d = S.pendulum()
    N = 2
    rp, rr, ang = S.initial_conditions(d, 1, 5)
    st1 = orc.default_qp(d, 1, rp, rr, ang)
    a1 = S.actions(d, 1, 3, 5).astype(np.float64)
    f1, n1 = orc.reverse_flops(d, st1, a1)
    f2, n2 = orc.reverse_flops(d, np.repeat(st1, N, axis=0), np.repeat(a1, N, axis=1))
    assert f2 == N * f1 and n2 == N * n1 and f1 > 0
    sb = S.SceneBuilder()
    sb.body("ball", 1.0, (0.4, 0.4, 0.4), (0, 0, 5.0))
    free = sb.build()
    st = orc.default_qp(free, 1, np.array([[0, 0, 5.0]]), None, None)
    one, _ = orc.reverse_flops(free, st, np.zeros((1, 1, 0)))
    three, _ = orc.reverse_flops(free, st, np.zeros((3, 1, 0)))
    assert three == 3 * one


# ----------------------------------------------------------------- two-body contacts, rotated anisotropic bodies
def two_body_scene(kind, mu=1.0, e=0.0, seed=0):
    """Two free bodies with distinct principal inertias, no gravity, no plane:
    capsule-capsule or capsule-box.  One substep per step (h = 5 ms)."""
    rng = np.random.default_rng(seed)
    sb = S.SceneBuilder(dt=0.005, substeps=1, gravity=(0, 0, 0))
    Ia = np.sort(rng.uniform(0.05, 0.6, size=3)) * [1.0, 1.7, 3.1]
    a = sb.capsule_body("a", 1.7, 0.12, 0.7, (0, 0, 0), (0, 0, 1), friction=mu, inertia=Ia)
    sb.colliders[-1]["elasticity"] = e
    if kind == "capsule":
        Ib = np.sort(rng.uniform(0.05, 0.6, size=3)) * [1.0, 2.3, 1.4]
        b = sb.capsule_body("b", 0.9, 0.09, 0.5, (0, 0, 0), (0, 0, 1), friction=1.0, inertia=Ib)
        cb = sb.collider_of(b)
    else:
        half = np.array([0.11, 0.07, 0.05])
        b = sb.body("b", 0.8, S.box_inertia(0.8, half) * [1.0, 1.3, 0.7], (0, 0, 0))
        cb = sb.collider(b, S.BOX, half=half, friction=1.0)
    sb.colliders[cb]["elasticity"] = 1.0
    sb.pair(sb.collider_of(a), cb)
    return sb.build()


def world_inv_inertia(q, inertia):
    R = rotmats(q)
    return R @ np.diag(1.0 / np.asarray(inertia)) @ R.T


def momenta(desc, x, q, v, w):
    """Linear and angular momentum (about the origin) computed here, from the
    state and the descriptor alone: sum m v and sum x × m v + R diag(I) R^T w."""
    P = np.zeros(3)
    L = np.zeros(3)
    for b in range(len(desc["mass"])):
        m = desc["mass"][b]
        R = rotmats(q[b])
        P += m * v[b]
        L += np.cross(x[b], m * v[b]) + R @ np.diag(desc["inertia"][b]) @ R.T @ w[b]
    return P, L


def touching_states(desc, rng, n_want):
    """Random generic poses and velocities of the two bodies with exactly one
    active contact after the kinematic integrator of the coming substep."""
    h = desc["dt"] / desc["substeps"]
    d1 = dict(desc, substeps=1, dt=h)
    out = []
    tries = 0
    while len(out) < n_want and tries < 20000:
        tries += 1
        st = np.zeros((1, 2, 13))
        for b in range(2):
            st[0, b, 3:7] = axis_angle(rng.normal(size=3), rng.uniform(0.3, 3.0))
            st[0, b, 7:10] = rng.normal(size=3) * 0.8
            st[0, b, 10:13] = rng.normal(size=3) * 2.0
        st[0, 0, 0:3] = rng.normal(size=3) * 0.05
        st[0, 1, 0:3] = st[0, 0, 0:3] + rng.normal(size=3) * 0.17
        post = orc.rollout(d1, st, np.zeros((1, 1, 0)))
        pk = st.copy()
        pk[0, :, 0:7] = post[0, :, 0:7]  # post-kinematic pose, pre-update velocities
        cts = orc.contacts(desc, pk[0])
        if len(cts) == 1 and cts[0][2] > 1e-4:
            out.append((st, post, cts[0]))
    assert len(out) == n_want, f"only {len(out)} touching configurations in {tries} tries"
    return out


@pytest.mark.parametrize("kind", ["capsule", "box"])
@pytest.mark.parametrize("elasticity", [0.0, 0.5])
def test_two_body_contact_conserves_momentum(kind, elasticity):
    """Sec. 7.2 contact between two free bodies, rotated and with anisotropic
    inertia (g = 0, no plane): the impulse is equal and opposite at one point,
    so one substep conserves sum m v to roundoff and sum x × m v +
    R diag(I) R^T w about the origin exactly (both taken at the post-kinematic
    pose, before and after the collision integrator).  A sign error on the
    second body, a swapped lever arm or a transposed world inertia breaks
    one of the two."""
    d = two_body_scene(kind, e=elasticity, seed=1)
    rng = np.random.default_rng(10 + (kind == "box") + 2 * int(elasticity * 2))
    n_moved = 0
    for st, post, ct in touching_states(d, rng, 25):
        x, q = post[0, :, 0:3], post[0, :, 3:7]
        P0, L0 = momenta(d, x, q, st[0, :, 7:10], st[0, :, 10:13])
        P1, L1 = momenta(d, x, q, post[0, :, 7:10], post[0, :, 10:13])
        scale = 1.0 + np.abs(P0).max() + np.abs(L0).max()
        assert np.abs(P1 - P0).max() < 1e-12 * scale
        assert np.abs(L1 - L0).max() < 1e-10 * scale
        n_moved += np.abs(post[0, :, 7:13] - st[0, :, 7:13]).max() > 1e-6
    assert n_moved >= 12  # the contacts really changed the velocities
    # several substeps in a row, each checked across its own collision update
    st = touching_states(d, np.random.default_rng(99), 1)[0][0]
    d1 = dict(d, substeps=1)
    for _ in range(12):
        post = orc.rollout(d1, st, np.zeros((1, 1, 0)))
        x, q = post[0, :, 0:3], post[0, :, 3:7]
        P0, L0 = momenta(d, x, q, st[0, :, 7:10], st[0, :, 10:13])
        P1, L1 = momenta(d, x, q, post[0, :, 7:10], post[0, :, 10:13])
        assert np.abs(P1 - P0).max() < 1e-12 * (1 + np.abs(P0).max())
        assert np.abs(L1 - L0).max() < 1e-10 * (1 + np.abs(L0).max())
        st = post


@pytest.mark.parametrize("kind", ["capsule", "box"])
def test_two_body_contact_velocity_changes(kind):
    """One substep with one contact: body a changes by dv = J/m_a and
    dw = R_a diag(1/I_a) R_a^T (l_a × J), body b by -J/m_b and
    -R_b diag(1/I_b) R_b^T (l_b × J), with l = p - x at the contact point p
    the oracle reports (Sec. 7.2; the world inverse inertia of Sec. 3 at the
    post-kinematic orientation).  Without friction the normal relative
    velocity afterwards is the Baumgarte/restitution target
    max(beta depth / h, -e u_n) (velocity-level contact), which pins the
    two-body effective mass."""
    for mu, e in ((1.0, 0.0), (0.0, 0.0), (0.0, 0.5)):
        d = two_body_scene(kind, mu=mu, e=e, seed=2)
        h = d["dt"] / d["substeps"]
        rng = np.random.default_rng(20 + (kind == "box"))
        n_active = 0
        for st, post, (ba, bb, depth, n, p) in touching_states(d, rng, 15):
            assert (ba, bb) == (0, 1)
            x, q = post[0, :, 0:3], post[0, :, 3:7]
            dv = post[0, :, 7:10] - st[0, :, 7:10]
            dw = post[0, :, 10:13] - st[0, :, 10:13]
            J = d["mass"][0] * dv[0]
            la, lb = p - x[0], p - x[1]
            assert np.allclose(dv[1], -J / d["mass"][1], atol=1e-13, rtol=0)
            assert np.allclose(dw[0], world_inv_inertia(q[0], d["inertia"][0]) @ np.cross(la, J), atol=1e-11, rtol=0)
            assert np.allclose(dw[1], -world_inv_inertia(q[1], d["inertia"][1]) @ np.cross(lb, J), atol=1e-11, rtol=0)
            u0 = (st[0, 0, 7:10] + np.cross(st[0, 0, 10:13], la)) - (st[0, 1, 7:10] + np.cross(st[0, 1, 10:13], lb))
            un0 = float(u0 @ n)
            jn = float(J @ n)
            if mu == 0.0:
                # no friction: the impulse is along n
                assert np.linalg.norm(J - jn * n) < 1e-12 * (1 + abs(jn))
                if jn > 0:
                    u1 = (post[0, 0, 7:10] + np.cross(post[0, 0, 10:13], la)) - \
                         (post[0, 1, 7:10] + np.cross(post[0, 1, 10:13], lb))
                    target = max(d["baumgarte"] / h * depth, -e * un0)
                    assert abs(float(u1 @ n) - target) < 1e-10 * (1 + abs(target))
                    n_active += 1
                else:  # separating faster than the target: no impulse
                    assert max(d["baumgarte"] / h * depth, -e * un0) <= un0 + 1e-12
            else:
                # Coulomb: the normal part pushes a off b, the tangential part is capped by mu j_n
                assert jn >= -1e-12
                assert np.linalg.norm(J - jn * n) <= mu * jn + 1e-10
        if mu == 0.0:
            assert n_active >= 5


# ----------------------------------------------------------------- environment layer (Sec. 4.2)
def test_env_oracle_observation_reward_done_closed_forms():
    """The environment layer's oracle (oracle/env.py) against closed forms: a
    child spinning freely about the hinge axis of a frozen parent (no springs
    acting, g = 0) turns by 2 atan(h w / 2) per substep, so its observed joint
    angle advances by that much per step and its observed rate is w; the root
    observation is the root's state; the reward of a frozen root is
    healthy - ctrl_cost * sum clamp(a)^2, and done follows the root height."""
    from oracle import env as oenv
    w, h, subs = 0.7, 0.01, 1
    d = hinge_system(gear=0.0, ca=0.0, I=0.8, ka=0.0, c=0.0, dt=h, substeps=subs)
    d["stiffness"] = np.zeros_like(d["stiffness"])
    st = state_of(d)
    st[0, 1, 10:13] = [w, 0.0, 0.0]  # about the hinge axis (world x)
    obs0 = oenv.observe(d, st)
    assert obs0.shape == (1, oenv.obs_size(d)) and oenv.obs_size(d) == 13
    spec = oenv.EnvSpec(forward_weight=2.0, healthy_reward=0.25, ctrl_cost=0.5, min_z=-1.0, max_z=1.0,
                        auto_reset=False)
    T = 6
    acts = np.full((T, 1, 1), 1.7)  # clamped to 1 for the cost
    sT, obs, rew, done = oenv.env_rollout(d, spec, st, st, acts)
    step = 2 * math.atan(h * w / 2)
    for t in range(T):
        assert abs(obs[t, 0, 11] - (obs0[0, 11] + (t + 1) * step)) < 1e-12
        assert abs(obs[t, 0, 12] - w) < 1e-12
        assert np.array_equal(obs[t, 0, :11], np.concatenate([[st[0, 0, 2]], st[0, 0, 3:13]]))
    assert np.allclose(rew, 0.25 - 0.5 * 1.0, atol=1e-15)  # frozen root: no progress
    assert not done.any()
    # done: a healthy range that excludes the root's height ends every step; the reset restores the state
    spec2 = oenv.EnvSpec(forward_weight=2.0, healthy_reward=0.25, ctrl_cost=0.5, min_z=0.5, max_z=1.0,
                         auto_reset=True)
    reset = st.copy()
    reset[0, 1, 10:13] = [-w, 0.0, 0.0]
    sT2, obs2, rew2, done2 = oenv.env_rollout(d, spec2, st, reset, acts)
    assert done2.all() and np.allclose(rew2, -0.5, atol=1e-15)
    assert abs(obs2[0, 0, 12] - w) < 1e-12 and abs(obs2[1, 0, 12] + w) < 1e-12  # restarted from the reset state


# ----------------------------------------------------------------- variants of the step
def test_global_damping_closed_form():
    """Global damping, no forces (g = 0): each substep scales v by
    (1 - h d_l) and w by (1 - h d_a), and x follows the discrete sum
    x_n = x0 + h v0 (1 - rho^n) / (1 - rho)."""
    d = single_body(inertia=(0.2, 0.9, 1.7))
    d["linear_damping"], d["angular_damping_global"] = 0.8, 1.3
    v0, w0, x0 = np.array([1.0, -2.0, 0.5]), np.array([0.3, 0.1, -0.7]), np.array([0.1, 0.2, 0.3])
    st = state_of(d, pos=x0, vel=v0, ang=w0)
    T = 4
    out = orc.rollout(d, st, np.zeros((T, 1, 0)))
    n, h = T * 10, 0.005
    rl, ra = 1 - h * 0.8, 1 - h * 1.3
    assert np.allclose(out[0, 0, 7:10], v0 * rl ** n, atol=1e-13, rtol=0)
    assert np.allclose(out[0, 0, 10:13], w0 * ra ** n, atol=1e-13, rtol=0)
    assert np.allclose(out[0, 0, 0:3], x0 + h * v0 * (1 - rl ** n) / (1 - rl), atol=1e-13, rtol=0)


def test_gyroscopic_term():
    """The gyroscopic torque -w x (I_w w): (1) it vanishes for an isotropic
    body; (2) one substep of a torque-free anisotropic body changes w by
    -h I_w^-1 (w x I_w w) at the post-kinematic orientation (computed here);
    (3) with it, a torque-free tumbling body keeps its angular momentum
    I_w w to O(h), without it (w constant) the momentum swings."""
    # (1)
    d = single_body(inertia=(0.7, 0.7, 0.7))
    st = state_of(d, quat=axis_angle([1, 2, 3], 0.9), ang=[1.0, -2.0, 3.0])
    a = np.zeros((3, 1, 0))
    on = orc.rollout(dict(d, gyroscopic=1), st, a)
    assert np.abs(on - orc.rollout(d, st, a)).max() < 1e-13
    # (2)
    I = np.array([0.2, 0.9, 1.7])
    d1 = single_body(inertia=tuple(I), dt=0.005, substeps=1)
    w0 = np.array([1.0, -2.0, 3.0])
    st = state_of(d1, quat=axis_angle([1, -1, 2], 0.7), ang=w0)
    out = orc.rollout(dict(d1, gyroscopic=1), st, np.zeros((1, 1, 0)))
    R = rotmats(out[0, 0, 3:7])
    Iw = R @ np.diag(I) @ R.T
    w1 = w0 - 0.005 * np.linalg.solve(Iw, np.cross(w0, Iw @ w0))
    assert np.allclose(out[0, 0, 10:13], w1, atol=1e-13, rtol=0)
    # (3)
    d = single_body(inertia=tuple(I), dt=0.05, substeps=40)
    st = state_of(d, quat=axis_angle([1, -1, 2], 0.7), ang=w0)

    def momentum(s):
        R = rotmats(s[0, 0, 3:7])
        return R @ np.diag(I) @ R.T @ s[0, 0, 10:13]

    L0 = momentum(st)
    drift = {}
    for g in (0, 1):
        s = orc.rollout(dict(d, gyroscopic=g), st, np.zeros((20, 1, 0)))  # 1 s
        drift[g] = np.linalg.norm(momentum(s) - L0) / np.linalg.norm(L0)
    assert drift[1] < 0.02 and drift[0] > 10 * drift[1], drift


def test_target_angle_actuator_converges_to_its_target():
    """A hinge driven by a target-angle actuator (frozen parent, no gravity,
    angular damping on): the action a picks theta* = (lo + hi)/2 + a (hi -
    lo)/2 in the limit range, and the joint settles at theta* (where the
    actuator's torque gear (theta* - theta) vanishes)."""
    sb = S.SceneBuilder(dt=0.01, substeps=4, gravity=(0, 0, 0))
    p = sb.body("P", 1.0, (1, 1, 1), (0, 0, 0), frozen_pos=(1, 1, 1), frozen_rot=(1, 1, 1))
    cb = sb.body("C", 1.0, (0.5, 0.5, 0.5), (0, 0, 0))
    j = sb.joint(p, cb, anchor=(0, 0, 0), axis=(1, 0, 0), ref=(0, 1, 0), stiffness=10000.0, spring_damping=5.0,
                 angular_stiffness=40.0, angular_damping=2.0, limits=((-40, 60),), limit_stiffness=50.0)
    sb.actuator(j, 0, 20.0, kind="angle")
    d = sb.build()
    assert list(d["act_type"]) == [1]
    st = state_of(d)
    for a in (-0.6, 0.25, 1.7):
        out = orc.rollout(d, st, np.full((1500, 1, 1), a))  # 15 s, about 30 decay times
        lo, hi = math.radians(-40), math.radians(60)
        target = 0.5 * (lo + hi) + 0.5 * (hi - lo) * min(max(a, -1), 1)
        assert abs(orc.joint_angles(d, out)[0, 0] - target) < 1e-6, a
        assert np.abs(out[0, 1, 10:13]).max() < 1e-6


def test_two_dof_joint_twist_spring_and_free_axes():
    """2-DOF (universal) joint, READING: rotations about its two joint axes
    meet no spring (inside the limits), the twist about the third axis is
    held by a spring of the alignment stiffness k_a.  Frozen parent, child
    centred on the anchor, g = 0, no damping; one substep from rest: a child
    turned by 0.3 rad about the first axis stays at rest, a child twisted by
    0.3 rad about the third axis gets w = -h k_a 0.3 / I along that axis."""
    h, I, ka = 0.005, 0.5, 40.0
    sb = S.SceneBuilder(dt=h, substeps=1, gravity=(0, 0, 0))
    p = sb.body("P", 1.0, (1, 1, 1), (0, 0, 0), frozen_pos=(1, 1, 1), frozen_rot=(1, 1, 1))
    cb = sb.body("C", 1.0, (I, I, I), (0, 0, 0))
    sb.joint(p, cb, anchor=(0, 0, 0), axis=(1, 0, 0), ref=(0, 1, 0), dof=2, stiffness=10000.0,
             spring_damping=0.0, angular_stiffness=ka, angular_damping=0.0, limits=((-60, 60), (-60, 60)),
             limit_stiffness=50.0)
    d = sb.build()
    assert list(d["dof"]) == [2]
    st = state_of(d)
    st[0, 1, 3:7] = axis_angle([1, 0, 0], 0.3)  # about joint axis 0 (world x)
    out = orc.rollout(d, st, np.zeros((1, 1, 0)))
    assert np.abs(out[0, 1, 7:13]).max() < 1e-14
    st[0, 1, 3:7] = axis_angle([0, 0, 1], 0.3)  # twist about the third axis (world z)
    assert abs(orc.joint_angles(d, st)[0, 0]) < 1e-15
    out = orc.rollout(d, st, np.zeros((1, 1, 0)))
    assert np.allclose(out[0, 1, 10:13], [0.0, 0.0, -h * ka * 0.3 / I], atol=1e-14, rtol=0)
    assert np.abs(out[0, 1, 7:10]).max() < 1e-14
