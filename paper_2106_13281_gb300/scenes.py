"""Seeded synthetic scenes and inputs.

This module is the one source of inputs that both the CUDA path and the FP64
oracle consume.  It holds scene *descriptions* (bodies, joints, actuators,
colliders, collision pairs - the system specification of Sec. 4.1 and App. A)
and seeded random inputs (actions, initial joint angles, root heights).  It
holds none of the step's arithmetic: no integration, no forces, no contacts
and no default_qp (both sides implement those on their own).

Descriptors are dicts of numpy arrays with the field names of the C
descriptor (``brax_desc`` in include/brax.h).  Angles in the descriptor are in
degrees (App. A ``angle_limit``); quaternions are (w, x, y, z); each body's
inertia is principal, in its own frame.

The scene geometry below - quadruped, biped, two-link pendulum, seven-hinge
arm with a box - is synthetic: the paper's own scene files are not part of it.
Shapes, masses, gears and sizes follow the workload descriptions (quadruped:
torso capsule r 0.25 len 0.5 mass 10, legs r 0.08 len 0.4 mass 1, hips +-30
deg, knees 30..70 deg, gear 150, friction 1, gravity -9.81, dt 0.05 with 10
substeps).
"""
from __future__ import annotations

import numpy as np

PLANE, CAPSULE, BOX = 0, 1, 2
STATE_SIZE = 13


# --------------------------------------------------------------------- geometry helpers
# Scene construction only: orientations of bodies and joint frames at the
# designed rest pose.
def quat_from_matrix(R):
    """Unit quaternion (w,x,y,z) of a proper rotation matrix (columns = body axes)."""
    R = np.asarray(R, dtype=np.float64)
    t = np.trace(R)
    if t > 0:
        s = np.sqrt(t + 1.0) * 2
        q = [0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s]
    elif R[0, 0] > R[1, 1] and R[0, 0] > R[2, 2]:
        s = np.sqrt(1.0 + R[0, 0] - R[1, 1] - R[2, 2]) * 2
        q = [(R[2, 1] - R[1, 2]) / s, 0.25 * s, (R[0, 1] + R[1, 0]) / s, (R[0, 2] + R[2, 0]) / s]
    elif R[1, 1] > R[2, 2]:
        s = np.sqrt(1.0 + R[1, 1] - R[0, 0] - R[2, 2]) * 2
        q = [(R[0, 2] - R[2, 0]) / s, (R[0, 1] + R[1, 0]) / s, 0.25 * s, (R[1, 2] + R[2, 1]) / s]
    else:
        s = np.sqrt(1.0 + R[2, 2] - R[0, 0] - R[1, 1]) * 2
        q = [(R[1, 0] - R[0, 1]) / s, (R[0, 2] + R[2, 0]) / s, (R[1, 2] + R[2, 1]) / s, 0.25 * s]
    q = np.array(q)
    q /= np.linalg.norm(q)
    return q if q[0] >= 0 else -q


def matrix_from_quat(q):
    w, x, y, z = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def frame_from_axes(x, y):
    """Rotation matrix with columns (x, y, x cross y) after orthonormalising y against x."""
    x = np.asarray(x, dtype=np.float64)
    x = x / np.linalg.norm(x)
    y = np.asarray(y, dtype=np.float64)
    y = y - x * np.dot(x, y)
    y = y / np.linalg.norm(y)
    return np.stack([x, y, np.cross(x, y)], axis=1)


def capsule_inertia(mass, radius, length):
    """Solid capsule (cylinder + two hemispheres, mass split by volume), axis z.
    `length` is tip to tip."""
    r = radius
    H = max(length - 2 * r, 0.0)
    v_cyl = np.pi * r * r * H
    v_hs = 4.0 / 3.0 * np.pi * r ** 3
    mc = mass * v_cyl / (v_cyl + v_hs)
    mh = mass * v_hs / (v_cyl + v_hs)
    iz = mc * r * r / 2 + mh * 2 * r * r / 5
    ix = mc * (r * r / 4 + H * H / 12) + mh * (2 * r * r / 5 + H * H / 4 + 3 * H * r / 8)
    return np.array([ix, ix, iz])


def box_inertia(mass, half):
    a, b, c = 2 * np.asarray(half, dtype=np.float64)
    return mass / 12.0 * np.array([b * b + c * c, a * a + c * c, a * a + b * b])


# --------------------------------------------------------------------- builder
class SceneBuilder:
    """Programmatic system specification (the Python form of App. A)."""

    def __init__(self, dt=0.05, substeps=10, gravity=(0.0, 0.0, -9.81), baumgarte=0.1, contact_eps=1e-6):
        self.dt, self.substeps = dt, substeps
        self.gravity = tuple(gravity)
        self.baumgarte, self.contact_eps = baumgarte, contact_eps
        self.bodies, self.joints, self.actuators, self.colliders, self.pairs = [], [], [], [], []
        self.names = {}

    # bodies -----------------------------------------------------------
    def body(self, name, mass, inertia, pos, R=None, frozen_pos=(0, 0, 0), frozen_rot=(0, 0, 0)):
        R = np.eye(3) if R is None else np.asarray(R, dtype=np.float64)
        self.bodies.append(dict(name=name, mass=float(mass), inertia=np.asarray(inertia, dtype=np.float64),
                                pos=np.asarray(pos, dtype=np.float64), R=R,
                                frozen_pos=frozen_pos, frozen_rot=frozen_rot))
        self.names[name] = len(self.bodies) - 1
        return len(self.bodies) - 1

    def capsule_body(self, name, mass, radius, length, pos, axis, up_hint=(0, 0, 1), friction=1.0, inertia=None,
                     **kw):
        """A body whose frame z axis runs along a capsule collider (so the
        capsule's principal inertia is diagonal in the body frame).  The
        inertia defaults to the solid capsule's."""
        axis = np.asarray(axis, dtype=np.float64)
        axis /= np.linalg.norm(axis)
        hint = np.asarray(up_hint, dtype=np.float64)
        if abs(np.dot(hint, axis)) > 0.9:
            hint = np.array([1.0, 0, 0]) if abs(axis[0]) < 0.9 else np.array([0, 1.0, 0])
        xb = hint - axis * np.dot(hint, axis)
        xb /= np.linalg.norm(xb)
        R = np.stack([xb, np.cross(axis, xb), axis], axis=1)
        I = capsule_inertia(mass, radius, length) if inertia is None else np.asarray(inertia, dtype=np.float64)
        b = self.body(name, mass, I, pos, R, **kw)
        self.collider(b, CAPSULE, radius=radius, length=length, friction=friction)
        return b

    # joints -----------------------------------------------------------
    def joint(self, parent, child, anchor, axis, ref, dof=1, stiffness=10000.0, spring_damping=10.0,
              angular_stiffness=100.0, angular_damping=0.2, limits=((-180, 180),), limit_stiffness=500.0):
        """Joint at world point `anchor` of the rest pose; `axis` is the hinge
        (joint frame x) and `ref` the joint frame y, both in world coordinates
        at rest.  For dof 3 the joint frame's x, y, z are the three axes."""
        P, Cb = self.bodies[parent], self.bodies[child]
        Fw = frame_from_axes(axis, ref)
        lo = np.zeros(3)
        hi = np.zeros(3)
        for i, (a, b) in enumerate(limits):
            lo[i], hi[i] = a, b
        self.joints.append(dict(
            parent=parent, child=child, dof=dof,
            parent_offset=P["R"].T @ (np.asarray(anchor) - P["pos"]),
            child_offset=Cb["R"].T @ (np.asarray(anchor) - Cb["pos"]),
            parent_frame=quat_from_matrix(P["R"].T @ Fw), child_frame=quat_from_matrix(Cb["R"].T @ Fw),
            stiffness=stiffness, spring_damping=spring_damping, angular_stiffness=angular_stiffness,
            angular_damping=angular_damping, limit_lo=lo, limit_hi=hi, limit_stiffness=limit_stiffness))
        return len(self.joints) - 1

    def actuator(self, joint, axis=0, gear=1.0, kind="torque"):
        """A torque actuator (torque = gear * clamp(a)), or with kind="angle" a
        target-angle actuator (a spring of stiffness gear toward the angle the
        action picks in the axis' limit range)."""
        assert kind in ("torque", "angle")
        self.actuators.append(dict(joint=joint, axis=axis, gear=float(gear), type=0 if kind == "torque" else 1))
        return len(self.actuators) - 1

    # colliders --------------------------------------------------------
    def collider(self, body, ctype, pos=(0, 0, 0), R=None, radius=0.0, length=0.0, half=(0, 0, 0),
                 friction=1.0, elasticity=0.0):
        R = np.eye(3) if R is None else np.asarray(R, dtype=np.float64)
        self.colliders.append(dict(body=body, type=ctype, pos=np.asarray(pos, dtype=np.float64),
                                   rot=quat_from_matrix(R), radius=radius, length=length,
                                   half=np.asarray(half, dtype=np.float64), friction=friction,
                                   elasticity=elasticity))
        return len(self.colliders) - 1

    def plane(self, point=(0, 0, 0), normal=(0, 0, 1), friction=1.0, elasticity=0.0):
        """A static plane (collider body -1); the collider frame's z axis is the normal."""
        n = np.asarray(normal, dtype=np.float64)
        n /= np.linalg.norm(n)
        helper = np.array([1.0, 0, 0]) if abs(n[0]) < 0.9 else np.array([0, 1.0, 0])
        x = np.cross(helper, n)
        x /= np.linalg.norm(x)
        R = np.stack([x, np.cross(n, x), n], axis=1)
        return self.collider(-1, PLANE, pos=point, R=R, friction=friction, elasticity=elasticity)

    def pair(self, a, b):
        self.pairs.append((a, b))

    def collider_of(self, body):
        for i, c in enumerate(self.colliders):
            if c["body"] == body:
                return i
        raise KeyError(body)

    # output -----------------------------------------------------------
    def build(self) -> dict:
        B, J, A, Cn, P = len(self.bodies), len(self.joints), len(self.actuators), len(self.colliders), len(self.pairs)
        f = lambda rows, k, w: np.array([r[k] for r in rows], dtype=np.float64).reshape(len(rows), w) if rows else np.zeros((0, w))
        d = dict(
            substeps=int(self.substeps), dt=float(self.dt), gravity=np.array(self.gravity, dtype=np.float64),
            baumgarte=float(self.baumgarte), contact_eps=float(self.contact_eps), average_contacts=1,
            mass=np.array([b["mass"] for b in self.bodies]),
            inertia=f(self.bodies, "inertia", 3),
            rest_pos=f(self.bodies, "pos", 3),
            rest_rot=np.array([quat_from_matrix(b["R"]) for b in self.bodies]).reshape(B, 4),
            frozen_pos=np.array([b["frozen_pos"] for b in self.bodies], dtype=np.uint8).reshape(B, 3),
            frozen_rot=np.array([b["frozen_rot"] for b in self.bodies], dtype=np.uint8).reshape(B, 3),
            parent=np.array([j["parent"] for j in self.joints], dtype=np.int32),
            child=np.array([j["child"] for j in self.joints], dtype=np.int32),
            dof=np.array([j["dof"] for j in self.joints], dtype=np.int32),
            parent_offset=f(self.joints, "parent_offset", 3), child_offset=f(self.joints, "child_offset", 3),
            parent_frame=f(self.joints, "parent_frame", 4), child_frame=f(self.joints, "child_frame", 4),
            stiffness=np.array([j["stiffness"] for j in self.joints], dtype=np.float64),
            spring_damping=np.array([j["spring_damping"] for j in self.joints], dtype=np.float64),
            angular_stiffness=np.array([j["angular_stiffness"] for j in self.joints], dtype=np.float64),
            angular_damping=np.array([j["angular_damping"] for j in self.joints], dtype=np.float64),
            limit_lo=f(self.joints, "limit_lo", 3), limit_hi=f(self.joints, "limit_hi", 3),
            limit_stiffness=np.array([j["limit_stiffness"] for j in self.joints], dtype=np.float64),
            act_joint=np.array([a["joint"] for a in self.actuators], dtype=np.int32),
            act_axis=np.array([a["axis"] for a in self.actuators], dtype=np.int32),
            gear=np.array([a["gear"] for a in self.actuators], dtype=np.float64),
            act_type=np.array([a["type"] for a in self.actuators], dtype=np.int32),
            col_body=np.array([c["body"] for c in self.colliders], dtype=np.int32),
            col_type=np.array([c["type"] for c in self.colliders], dtype=np.int32),
            col_pos=f(self.colliders, "pos", 3), col_rot=f(self.colliders, "rot", 4),
            radius=np.array([c["radius"] for c in self.colliders], dtype=np.float64),
            length=np.array([c["length"] for c in self.colliders], dtype=np.float64),
            half_extents=f(self.colliders, "half", 3),
            friction=np.array([c["friction"] for c in self.colliders], dtype=np.float64),
            elasticity=np.array([c["elasticity"] for c in self.colliders], dtype=np.float64),
            pair_a=np.array([p[0] for p in self.pairs], dtype=np.int32),
            pair_b=np.array([p[1] for p in self.pairs], dtype=np.int32),
            body_names=[b["name"] for b in self.bodies],
        )
        assert d["rest_rot"].shape == (B, 4) and d["frozen_pos"].shape == (B, 3)
        assert P == len(d["pair_a"]) and Cn == len(d["col_body"]) and A == len(d["gear"]) and J == len(d["parent"])
        return d


def n_dof(desc) -> int:
    return int(np.sum(desc["dof"])) if len(desc["dof"]) else 0


# --------------------------------------------------------------------- joint constants
# The paper prints only the App. A stiffness (10000); it states that spring
# joints need tuning of damping, mass scale and step size (Sec. 7.1).  The
# values below were chosen per scene with the explicit integrator's stability
# bound (h^2 k w + 2 h c w < 4 for inverse effective mass w) and checked by
# oracle rollouts under random actions.
QUADRUPED_JOINT = dict(stiffness=10000.0, spring_damping=30.0, angular_stiffness=1000.0, angular_damping=10.0,
                       limit_stiffness=1000.0)

# Inertia of jointed bodies: App. A gives its 1 kg bodies a unit diagonal
# inertia, and Sec. 7.1 / App. D name mass and inertia scale among what spring
# joints need tuned.  With solid-shape inertia (about 0.012 kg m^2 for a 1 kg,
# 0.4 m leg) a 150 N m actuator adds about 63 rad/s per 5 ms substep, beyond
# what an explicit spring-damper joint can hold; the jointed bodies of the
# scenes below therefore use the App. A value (1, 1, 1) kg m^2.
UNIT_INERTIA = (1.0, 1.0, 1.0)


# --------------------------------------------------------------------- scenes
def appendix_a() -> dict:
    """The example system of App. A: a frozen parent and a 1 kg child joined
    by one joint of stiffness 10000 with child_offset z = 1, limits -180..180
    (the text form; the programmatic listing's `min = 180` is read as a typo),
    dt 0.01, 1 substep, gravity -9.8."""
    sb = SceneBuilder(dt=0.01, substeps=1, gravity=(0, 0, -9.8))
    p = sb.body("Parent", 1.0, (1, 1, 1), (0, 0, 0), frozen_pos=(1, 1, 1), frozen_rot=(1, 1, 1))
    c = sb.body("Child", 1.0, (1, 1, 1), (0, 0, -1.0))
    sb.joint(p, c, anchor=(0, 0, 0), axis=(1, 0, 0), ref=(0, 1, 0), stiffness=10000.0, spring_damping=10.0,
             angular_stiffness=100.0, angular_damping=1.0, limits=((-180, 180),), limit_stiffness=100.0)
    return sb.build()


def quadruped(joint=None) -> dict:
    """9-body quadruped: torso capsule (r 0.25, len 0.5 -> a sphere, mass 10)
    and 4 legs x 2 capsule segments (r 0.08, len 0.4, mass 1).  Leg k leaves
    the torso at azimuth 45 + 90 k deg; hip axis z (limits +-30 deg), knee axis
    z x d (limits 30..70 deg: + bends the shin down).  8 torque actuators with
    gear 150; capsule-plane contacts only, friction 1."""
    jc = dict(QUADRUPED_JOINT if joint is None else joint)
    sb = SceneBuilder(dt=0.05, substeps=10, gravity=(0, 0, -9.81))
    torso_z = 0.75
    t = sb.body("torso", 10.0, UNIT_INERTIA, (0, 0, torso_z))
    sb.collider(t, CAPSULE, radius=0.25, length=0.5, friction=1.0)
    ground = sb.plane(friction=1.0)
    sb.pair(sb.collider_of(t), ground)
    ez = np.array([0.0, 0, 1])
    for k in range(4):
        phi = np.deg2rad(45 + 90 * k)
        d = np.array([np.cos(phi), np.sin(phi), 0.0])
        base = np.array([0, 0, torso_z])
        hip = base + 0.25 * d
        knee = hip + 0.4 * d
        th = sb.capsule_body(f"thigh{k}", 1.0, 0.08, 0.4, hip + 0.2 * d, d, inertia=UNIT_INERTIA)
        sh = sb.capsule_body(f"shin{k}", 1.0, 0.08, 0.4, knee + 0.2 * d, d, inertia=UNIT_INERTIA)
        jh = sb.joint(t, th, hip, axis=ez, ref=d, limits=((-30, 30),), **jc)
        jk = sb.joint(th, sh, knee, axis=np.cross(ez, d), ref=d, limits=((30, 70),), **jc)
        sb.actuator(jh, 0, 150.0)
        sb.actuator(jk, 0, 150.0)
        sb.pair(sb.collider_of(th), ground)
        sb.pair(sb.collider_of(sh), ground)
    return sb.build()


def biped(joint=None) -> dict:
    """17-capsule biped: torso, pelvis, head, 2 x (upper arm, forearm, hand),
    2 x (thigh, shin, foot, toe).  Neck, abdomen, shoulders and hips are
    3-axis joints; elbows, wrists, knees, ankles and toes are hinges
    (6 x 3 + 10 = 28 DOF, 28 actuators).  Capsule-plane contacts for every
    capsule and capsule-capsule self-collision on all 120 non-adjacent pairs."""
    base = dict(QUADRUPED_JOINT)
    if joint:
        base.update(joint)
    sb = SceneBuilder(dt=0.05, substeps=10, gravity=(0, 0, -9.81))
    up = (0, 0, 1.0)
    fx = (1.0, 0, 0)
    torso = sb.capsule_body("torso", 8.0, 0.10, 0.44, (0, 0, 1.28), up, up_hint=fx, inertia=UNIT_INERTIA)
    pelvis = sb.capsule_body("pelvis", 4.0, 0.09, 0.32, (0, 0, 0.97), (0, 1.0, 0), inertia=UNIT_INERTIA)
    head = sb.capsule_body("head", 2.0, 0.09, 0.20, (0, 0, 1.63), up, up_hint=fx, inertia=UNIT_INERTIA)
    X, Y, Z = np.eye(3)
    j3 = lambda p, c, a, lim, **kw: sb.joint(p, c, a, axis=X, ref=Y, dof=3, limits=lim, **{**base, **kw})
    j1 = lambda p, c, a, lim, **kw: sb.joint(p, c, a, axis=Y, ref=Z, dof=1, limits=(lim,), **{**base, **kw})
    neck = j3(torso, head, (0, 0, 1.52), ((-30, 30), (-30, 30), (-45, 45)))
    abdomen = j3(torso, pelvis, (0, 0, 1.06), ((-35, 35), (-45, 30), (-35, 35)))
    acts = [(neck, 3, 25.0), (abdomen, 3, 100.0)]
    for side, sy in (("l", 1.0), ("r", -1.0)):
        ya = 0.27 * sy
        ua = sb.capsule_body(f"upper_arm_{side}", 1.5, 0.045, 0.30, (0, ya, 1.30), up, up_hint=fx, inertia=UNIT_INERTIA)
        fa = sb.capsule_body(f"forearm_{side}", 1.0, 0.04, 0.28, (0, ya, 1.01), up, up_hint=fx, inertia=UNIT_INERTIA)
        ha = sb.capsule_body(f"hand_{side}", 0.5, 0.04, 0.12, (0, ya, 0.81), up, up_hint=fx, inertia=UNIT_INERTIA)
        sh = j3(torso, ua, (0, ya, 1.45), ((-60, 60), (-85, 60), (-45, 45)))
        el = j1(ua, fa, (0, ya, 1.15), (-150, 2))
        wr = j1(fa, ha, (0, ya, 0.87), (-60, 60))
        acts += [(sh, 3, 60.0), (el, 1, 40.0), (wr, 1, 15.0)]
    for side, sy in (("l", 1.0), ("r", -1.0)):
        yl = 0.10 * sy
        th = sb.capsule_body(f"thigh_{side}", 4.0, 0.07, 0.45, (0, yl, 0.695), up, up_hint=fx, inertia=UNIT_INERTIA)
        sn = sb.capsule_body(f"shin_{side}", 2.5, 0.05, 0.38, (0, yl, 0.28), up, up_hint=fx, inertia=UNIT_INERTIA)
        ft = sb.capsule_body(f"foot_{side}", 1.0, 0.04, 0.16, (0.06, yl, 0.045), fx, up_hint=up, inertia=UNIT_INERTIA)
        to = sb.capsule_body(f"toe_{side}", 0.5, 0.04, 0.10, (0.19, yl, 0.045), fx, up_hint=up, inertia=UNIT_INERTIA)
        hp = j3(pelvis, th, (0, yl, 0.92), ((-30, 30), (-100, 20), (-35, 35)))
        kn = j1(th, sn, (0, yl, 0.47), (-2, 150))
        an = j1(sn, ft, (0, yl, 0.09), (-45, 45))
        toe = j1(ft, to, (0.15, yl, 0.045), (-45, 45))
        acts += [(hp, 3, 100.0), (kn, 1, 100.0), (an, 1, 50.0), (toe, 1, 15.0)]
    for j, ndof, g in acts:
        for a in range(ndof):
            sb.actuator(j, a, g)
    ground = sb.plane(friction=1.0)
    B = len(sb.bodies)
    for b in range(B):
        sb.pair(sb.collider_of(b), ground)
    adjacent = {(j["parent"], j["child"]) for j in sb.joints} | {(j["child"], j["parent"]) for j in sb.joints}
    for a in range(B):
        for b in range(a + 1, B):
            if (a, b) not in adjacent:
                sb.pair(sb.collider_of(a), sb.collider_of(b))
    return sb.build()


def pendulum(joint=None) -> dict:
    """2-link capsule pendulum chain hanging from a frozen anchor (3 bodies,
    2 hinges about y, 2 actuators, capsule-plane contacts)."""
    jc = dict(stiffness=10000.0, spring_damping=10.0, angular_stiffness=300.0, angular_damping=2.0,
              limit_stiffness=300.0)
    if joint:
        jc.update(joint)
    sb = SceneBuilder(dt=0.05, substeps=10, gravity=(0, 0, -9.81))
    anchor = sb.body("anchor", 1.0, UNIT_INERTIA, (0, 0, 1.2), frozen_pos=(1, 1, 1), frozen_rot=(1, 1, 1))
    down = (0, 0, -1.0)
    l1 = sb.capsule_body("link1", 1.0, 0.05, 0.5, (0, 0, 0.95), down, up_hint=(1, 0, 0), inertia=UNIT_INERTIA)
    l2 = sb.capsule_body("link2", 1.0, 0.05, 0.5, (0, 0, 0.45), down, up_hint=(1, 0, 0), inertia=UNIT_INERTIA)
    j1 = sb.joint(anchor, l1, (0, 0, 1.2), axis=(0, 1, 0), ref=(0, 0, -1), limits=((-180, 180),), **jc)
    j2 = sb.joint(l1, l2, (0, 0, 0.7), axis=(0, 1, 0), ref=(0, 0, -1), limits=((-150, 150),), **jc)
    sb.actuator(j1, 0, 20.0)
    sb.actuator(j2, 0, 20.0)
    ground = sb.plane(friction=1.0)
    sb.pair(sb.collider_of(l1), ground)
    sb.pair(sb.collider_of(l2), ground)
    return sb.build()


def arm_box(joint=None) -> dict:
    """7-hinge capsule arm on a frozen base next to a 0.1 m box (mass 0.5)
    resting on the plane: capsule-plane, box-plane and capsule-box contacts."""
    jc = dict(stiffness=5000.0, spring_damping=10.0, angular_stiffness=300.0, angular_damping=2.0,
              limit_stiffness=300.0)
    if joint:
        jc.update(joint)
    sb = SceneBuilder(dt=0.05, substeps=10, gravity=(0, 0, -9.81))
    base = sb.body("base", 5.0, UNIT_INERTIA, (0, 0, 0.05), frozen_pos=(1, 1, 1), frozen_rot=(1, 1, 1))
    up = (0, 0, 1.0)
    axes = [(0, 0, 1), (0, 1, 0), (1, 0, 0), (0, 1, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    refs = [(1, 0, 0), (0, 0, 1), (0, 0, 1), (0, 0, 1), (0, 0, 1), (0, 0, 1), (1, 0, 0)]
    lims = [(-180, 180), (-90, 90), (-90, 90), (-120, 120), (-90, 90), (-120, 120), (-180, 180)]
    L = 0.22
    prev = base
    links = []
    for k in range(7):
        z0 = 0.1 + L * k
        lk = sb.capsule_body(f"link{k + 1}", 0.5, 0.04, L, (0, 0, z0 + L / 2), up, up_hint=(1, 0, 0), inertia=UNIT_INERTIA)
        jk = sb.joint(prev, lk, (0, 0, z0), axis=axes[k], ref=refs[k], limits=(lims[k],), **jc)
        sb.actuator(jk, 0, 20.0)
        links.append(lk)
        prev = lk
    half = (0.05, 0.05, 0.05)
    box = sb.body("box", 0.5, box_inertia(0.5, half), (0.35, 0.0, 0.05))
    bc = sb.collider(box, BOX, half=half, friction=1.0)
    ground = sb.plane(friction=1.0)
    for lk in links:
        sb.pair(sb.collider_of(lk), ground)
    sb.pair(bc, ground)
    for lk in links:
        sb.pair(sb.collider_of(lk), bc)
    return sb.build()


SCENES = dict(quadruped=quadruped, biped=biped, pendulum=pendulum, arm_box=arm_box, appendix_a=appendix_a)


# --------------------------------------------------------------------- seeded inputs
def planar(desc, axis=1) -> dict:
    """The planar masking of App. E (Halfcheetah): every body's position is
    frozen along world axis `axis` and its rotation about the other two, so
    motion stays in the plane normal to `axis` and turns only about it."""
    d = dict(desc)
    fp = np.array(desc["frozen_pos"], dtype=np.uint8).copy()
    fr = np.array(desc["frozen_rot"], dtype=np.uint8).copy()
    fp[:, axis] = 1
    for k in range(3):
        if k != axis:
            fr[:, k] = 1
    d["frozen_pos"], d["frozen_rot"] = fp, fr
    return d


def quadruped_variants() -> dict:
    """The quadruped with the variants of the step switched on: target-angle
    actuators at the knees (torque actuators at the hips), global linear and
    angular damping, the gyroscopic torque, and an anisotropic torso inertia
    (so that the gyroscopic term does not vanish)."""
    d = quadruped()
    d = dict(d)
    n_act = len(d["act_joint"])
    # joints alternate hip, knee per leg: knees are the children of thighs
    knee = np.array([d["parent"][j] != 0 for j in d["act_joint"]], dtype=bool)
    d["act_type"] = np.where(knee, 1, 0).astype(np.int32)
    d["gear"] = np.where(knee, 200.0, np.asarray(d["gear"], dtype=np.float64))
    d["linear_damping"] = 0.2
    d["angular_damping_global"] = 0.5
    d["gyroscopic"] = 1
    inertia = np.array(d["inertia"], dtype=np.float64).copy()
    inertia[0] = [0.8, 1.2, 1.6]
    d["inertia"] = inertia
    assert n_act == len(d["act_type"])
    return d


def quadruped_aniso() -> dict:
    """The quadruped with anisotropic inertias (torso and thighs) and nothing
    else changed: a hinge-only system whose reverse pass must carry the
    adjoint of the world inverse inertia I_w = R diag(1/I) R^T into the
    orientation (Sec. 3), which isotropic bodies do not exercise."""
    d = dict(quadruped())
    inertia = np.array(d["inertia"], dtype=np.float64).copy()
    inertia[0] = [0.8, 1.2, 1.6]
    for b, name in enumerate(d["body_names"]):
        if name.startswith("thigh"):
            inertia[b] = [1.3, 0.9, 1.1]
    d["inertia"] = inertia
    return d


def quadruped_2dof() -> dict:
    """The quadruped with 2-DOF (universal) hips: axis 0 swings the leg about
    the vertical (+-30 deg), axis 1 lifts it about the horizontal axis across
    the leg (+-20 deg); the twist about the leg is held by the joint's
    alignment spring.  12 torque actuators (gear 150)."""
    sb = SceneBuilder(dt=0.05, substeps=10, gravity=(0, 0, -9.81))
    jc = dict(QUADRUPED_JOINT)
    torso_z = 0.75
    t = sb.body("torso", 10.0, UNIT_INERTIA, (0, 0, torso_z))
    sb.collider(t, CAPSULE, radius=0.25, length=0.5, friction=1.0)
    ground = sb.plane(friction=1.0)
    sb.pair(sb.collider_of(t), ground)
    ez = np.array([0.0, 0, 1])
    for k in range(4):
        phi = np.deg2rad(45 + 90 * k)
        d = np.array([np.cos(phi), np.sin(phi), 0.0])
        hip = np.array([0, 0, torso_z]) + 0.25 * d
        knee = hip + 0.4 * d
        th = sb.capsule_body(f"thigh{k}", 1.0, 0.08, 0.4, hip + 0.2 * d, d, inertia=UNIT_INERTIA)
        sh = sb.capsule_body(f"shin{k}", 1.0, 0.08, 0.4, knee + 0.2 * d, d, inertia=UNIT_INERTIA)
        jh = sb.joint(t, th, hip, axis=ez, ref=np.cross(ez, d), dof=2, limits=((-30, 30), (-20, 20)), **jc)
        jk = sb.joint(th, sh, knee, axis=np.cross(ez, d), ref=d, limits=((30, 70),), **jc)
        sb.actuator(jh, 0, 150.0)
        sb.actuator(jh, 1, 150.0)
        sb.actuator(jk, 0, 150.0)
        sb.pair(sb.collider_of(th), ground)
        sb.pair(sb.collider_of(sh), ground)
    return sb.build()


def joint_angle_centres(desc) -> np.ndarray:
    """Per-DOF centre of the initial angle distribution (radians): 0 where 0
    lies inside the limit range, else the midpoint of the range (the knees)."""
    out = []
    for j in range(len(desc["dof"])):
        for a in range(int(desc["dof"][j])):
            lo, hi = desc["limit_lo"][j][a], desc["limit_hi"][j][a]
            out.append(0.0 if lo <= 0.0 <= hi else np.deg2rad(0.5 * (lo + hi)))
    return np.array(out)


def initial_conditions(desc, n_envs, seed, height_jitter=0.0, angle_sigma=0.1):
    """Seeded root poses and joint angles for default_qp: body 0 at its rest
    position with z + U(0, height_jitter), identity rotation, joint angles
    centre + N(0, angle_sigma^2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    root_pos = np.repeat(desc["rest_pos"][0][None, :], n_envs, axis=0).astype(np.float64)
    if height_jitter > 0:
        root_pos[:, 2] += rng.uniform(0.0, height_jitter, size=n_envs)
    root_rot = np.repeat(desc["rest_rot"][0][None, :], n_envs, axis=0).astype(np.float64)
    D = n_dof(desc)
    angles = joint_angle_centres(desc)[None, :] + rng.normal(0.0, angle_sigma, size=(n_envs, D))
    return root_pos, root_rot, angles


def actions(desc, n_envs, T, seed, low=-1.0, high=1.0) -> np.ndarray:
    """Seeded actions uniform[low, high], [T, N, A], float32."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    A = len(desc["gear"])
    return rng.uniform(low, high, size=(T, n_envs, A)).astype(np.float32)


def capsule_on_box(inside=False) -> dict:
    """Test scene for capsule-box contact: a 0.1 m box (mass 0.5) on the plane
    and a free capsule (r 0.04, len 0.3, mass 0.3) lying across its top
    face, tilted; with `inside` the capsule starts with its segment inside
    the box (the deep-penetration branch)."""
    sb = SceneBuilder(dt=0.05, substeps=10, gravity=(0, 0, -9.81))
    half = (0.05, 0.05, 0.05)
    box = sb.body("box", 0.5, box_inertia(0.5, half), (0.0, 0.0, 0.05))
    bc = sb.collider(box, BOX, half=half, friction=1.0)
    z = 0.06 if inside else 0.135
    axis = np.array([1.0, 0.3, 0.15])
    cap = sb.capsule_body("rod", 0.3, 0.04, 0.3, (0.02, 0.01, z), axis / np.linalg.norm(axis))
    ground = sb.plane(friction=1.0)
    sb.pair(bc, ground)
    sb.pair(sb.collider_of(cap), ground)
    sb.pair(sb.collider_of(cap), bc)
    return sb.build()


SCENES["capsule_on_box"] = lambda joint=None: capsule_on_box(False)
SCENES["capsule_in_box"] = lambda joint=None: capsule_on_box(True)
SCENES["quadruped_variants"] = lambda joint=None: quadruped_variants()
SCENES["quadruped_planar"] = lambda joint=None: planar(quadruped())
SCENES["quadruped_2dof"] = lambda joint=None: quadruped_2dof()
SCENES["quadruped_aniso"] = lambda joint=None: quadruped_aniso()
