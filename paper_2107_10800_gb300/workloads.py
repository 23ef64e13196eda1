"""Seeded synthetic workloads for the articulated-body solver.

This module only draws random numbers and lays out geometry (blob templates,
body centres, joint points, sliding schedules).  It holds none of the
method's arithmetic: no rotation matrices, no mobility, no constraint
Jacobians.  Both the CUDA path and the CPU oracle read the same dictionaries
from here.

Every workload is a dict with
  eta, a             viscosity and blob radius
  wall               0 free space, 1 no-slip wall at z = 0
  q      (M, 3)      body tracking points (lab frame)
  theta  (M, 4)      unit quaternions [s, p] (Sec. 2.1)
  blob_offset (M+1,) CSR offsets of each body's blobs
  rho    (Nb, 3)     body-frame blob offsets from the tracking point
  F      (M, 6)      external force and torque per body
  assembly (M,)      articulated-body index of each body
  body_p, body_q (P,) linked bodies of each link
and one of
  joints (P, 3)      lab-frame joint point of each passive link at the
                     initial pose (the body-frame vectors follow from it)
  dl(t) -> (dl_p, dl_q, dl_p_dot, dl_q_dot)
                     body-frame link vectors and their time derivatives for
                     time-dependent (active) links
"""
import math
import numpy as np

GOLDEN = (1.0 + 5.0 ** 0.5) / 2.0


def icosahedron(radius):
    """The 12 vertices (0, +-1, +-phi) and cyclic permutations, scaled to
    ``radius`` (the 12-blob shell used for the settling-filament bodies,
    Sec. 3.2.1)."""
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v.append((0.0, s1, s2 * GOLDEN))
            v.append((s1, s2 * GOLDEN, 0.0))
            v.append((s2 * GOLDEN, 0.0, s1))
    v = np.array(v, dtype=np.float64)
    return v * (radius / np.sqrt(1.0 + GOLDEN ** 2))


def _random_unit_quaternions(rng, n):
    """Uniformly distributed rotations: normalised 4-D Gaussians, s >= 0."""
    g = rng.standard_normal((n, 4))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    g[g[:, 0] < 0] *= -1.0
    return g


def _unit_vector(rng):
    g = rng.standard_normal(3)
    return g / np.linalg.norm(g)


def chains_free_space(seed, n_chains=4, bodies_per_chain=8, a=0.1,
                      shell_radius=0.5, step=1.05, box=10.0, eta=1.0):
    """Chains of icosahedral 12-blob shells joined by ball joints at the
    midpoints of neighbouring centres, free space.

    Centres follow a seeded random walk of fixed step inside a cube (a step
    that would leave the cube is redrawn); orientations are uniformly random;
    each body gets a force and torque with N(0, 1) components.  With the
    defaults: 32 bodies, 384 blobs, 28 links (1,428 unknowns).
    """
    rng = np.random.default_rng(np.random.Philox(seed))
    ico = icosahedron(shell_radius)
    q = []
    body_p, body_q, joints = [], [], []
    assembly = []
    for c in range(n_chains):
        x = rng.uniform(0.0, box, 3)
        for k in range(bodies_per_chain):
            if k > 0:
                while True:
                    cand = x + step * _unit_vector(rng)
                    if np.all(cand >= 0.0) and np.all(cand <= box):
                        break
                x = cand
            q.append(x.copy())
            assembly.append(c)
            idx = len(q) - 1
            if k > 0:
                body_p.append(idx - 1)
                body_q.append(idx)
                joints.append(0.5 * (q[idx - 1] + q[idx]))
    M = len(q)
    theta = _random_unit_quaternions(rng, M)
    F = rng.standard_normal((M, 6))
    rho = np.tile(ico, (M, 1))
    blob_offset = np.arange(M + 1, dtype=np.int64) * 12
    return dict(name="chains_free_space", eta=eta, a=a, wall=0,
                q=np.array(q), theta=theta, blob_offset=blob_offset, rho=rho,
                F=F, assembly=np.array(assembly, dtype=np.int64),
                body_p=np.array(body_p, dtype=np.int64),
                body_q=np.array(body_q, dtype=np.int64),
                joints=np.array(joints), dl=None)


def rod_template(nx=40, ny=2, spacing=0.2):
    """Blob grid of a rectangular rod in its body x-y plane, centred."""
    xs = (np.arange(nx) - 0.5 * (nx - 1)) * spacing
    ys = (np.arange(ny) - 0.5 * (ny - 1)) * spacing
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)


def diatom_colony(seed, n_rods=32, nx=40, ny=2, spacing=0.2, a=0.1,
                  stack=0.4, hmin=0.5, hmax=1.5, eta=1.0):
    """Colony of stacked rectangular rods above a no-slip wall, adjacent rods
    joined by two links that keep them parallel and let them slide
    (Sec. 5.1, Eq. const_bacillaria, generalised to an arbitrary fixed offset
    between the rods).

    Rods are parallel to the lab x-axis at t = 0 (identity orientations, so
    body and lab frames coincide then), stacked along y with spacing
    ``stack``, each at a seeded height in [hmin, hmax].  With
    d = q_q - q_p at t = 0 and sliding length L(t):
        dl_1p = d/2 + (L/2) e_x,  dl_1q = -dl_1p,
        dl_2p = d + L e_x,        dl_2q = 0.
    The sliding velocity of pair k is dL/dt = sin(2 pi t + phi_k) with seeded
    phases, so L(t) = (cos phi_k - cos(2 pi t + phi_k)) / (2 pi), L(0) = 0.
    With the defaults: 32 rods, 2,560 blobs, 62 links.
    """
    rng = np.random.default_rng(np.random.Philox(seed))
    tmpl = rod_template(nx, ny, spacing)
    heights = rng.uniform(hmin, hmax, n_rods)
    q = np.zeros((n_rods, 3))
    q[:, 1] = np.arange(n_rods) * stack
    q[:, 2] = heights
    theta = np.zeros((n_rods, 4))
    theta[:, 0] = 1.0
    phases = rng.uniform(0.0, 2.0 * math.pi, n_rods - 1)
    d = q[1:] - q[:-1]
    body_p, body_q = [], []
    for k in range(n_rods - 1):
        body_p += [k, k]
        body_q += [k + 1, k + 1]
    P = len(body_p)
    ex = np.array([1.0, 0.0, 0.0])

    def dl(t):
        L = (np.cos(phases) - np.cos(2 * math.pi * t + phases)) / (2 * math.pi)
        Ld = np.sin(2 * math.pi * t + phases)
        dl_p = np.zeros((P, 3)); dl_q = np.zeros((P, 3))
        dlp_dot = np.zeros((P, 3)); dlq_dot = np.zeros((P, 3))
        dl_p[0::2] = 0.5 * d + 0.5 * L[:, None] * ex
        dl_q[0::2] = -dl_p[0::2]
        dl_p[1::2] = d + L[:, None] * ex
        dlp_dot[0::2] = 0.5 * Ld[:, None] * ex
        dlq_dot[0::2] = -dlp_dot[0::2]
        dlp_dot[1::2] = Ld[:, None] * ex
        return dl_p, dl_q, dlp_dot, dlq_dot

    return dict(name="diatom_colony", eta=eta, a=a, wall=1, q=q, theta=theta,
                blob_offset=np.arange(n_rods + 1, dtype=np.int64) * (nx * ny),
                rho=np.tile(tmpl, (n_rods, 1)), F=np.zeros((n_rods, 6)),
                assembly=np.zeros(n_rods, dtype=np.int64),
                body_p=np.array(body_p, dtype=np.int64),
                body_q=np.array(body_q, dtype=np.int64),
                joints=None, dl=dl, phases=phases)


def batched_chains(seed, n_systems=256, lo=500, hi=20_000, a=0.1, eta=1.0):
    """Independent free-space suspensions of chains (the batched form): blob
    counts drawn log-uniform in [lo, hi] from the seed, rounded to whole
    12-blob icosahedral bodies, bodies in chains of 8 (the last chain of a
    suspension shorter) joined by ball joints, each suspension in a cube whose
    side keeps the body density of chains_free_space (32 bodies in a cube of
    side 10).  Returns a list of workload dicts."""
    rng = np.random.default_rng(np.random.Philox(seed))
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), n_systems))
    out = []
    for k, nb in enumerate(sizes):
        M = max(2, int(round(nb / 12.0)))
        n_chains = (M + 7) // 8
        w = chains_free_space(seed * 100003 + k, n_chains=n_chains, bodies_per_chain=8, a=a,
                              box=10.0 * (M / 32.0) ** (1.0 / 3.0), eta=eta)
        # trim to exactly M bodies (drop the tail of the last chain)
        keep = M
        w["q"] = w["q"][:keep]
        w["theta"] = w["theta"][:keep]
        w["F"] = w["F"][:keep]
        w["rho"] = w["rho"][:12 * keep]
        w["blob_offset"] = w["blob_offset"][:keep + 1]
        w["assembly"] = w["assembly"][:keep]
        lk = (w["body_p"] < keep) & (w["body_q"] < keep)
        w["body_p"], w["body_q"], w["joints"] = w["body_p"][lk], w["body_q"][lk], w["joints"][lk]
        w["name"] = "batched_chains[%d]" % k
        out.append(w)
    return out


def _fibonacci_ellipsoid(n, axes):
    """n quasi-uniform points on an ellipsoid (Fibonacci lattice on the unit
    sphere, stretched along the axes)."""
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    p = np.stack([z, r * np.cos(phi), r * np.sin(phi)], axis=1)
    return p * np.asarray(axes)


def bacterium_template(a=0.05, head_blobs=200, axes=(1.0, 0.5, 0.5),
                       n_seg=16, seg_blobs=10, pitch=1.5, radius=0.25):
    """Body-frame geometry of one bacterium: an ellipsoidal head (long axis
    along x) and a helical flagellum of rigid segments along -x, blobs spaced
    2a along the helix arc (Sec. 4.3 and 5.2 give the head-flagellum model).

    Returns (list of blob arrays in the bacterium frame, hinge points,
    segment joint points).  The hinge is two links on the helix axis, the
    pattern of the two-link head-flagellum joint in Sec. 4.3: one at the
    attachment point, one further along the axis.
    """
    head = _fibonacci_ellipsoid(head_blobs, axes)
    n_fl = n_seg * seg_blobs
    ds = 2.0 * a
    dtheta = ds / math.sqrt(radius ** 2 + (pitch / (2 * math.pi)) ** 2)
    x0 = -(axes[0] + a + radius)  # attachment a little behind the head
    ang = np.arange(n_fl) * dtheta
    fl = np.stack([x0 - pitch * ang / (2 * math.pi),
                   radius * np.cos(ang), radius * np.sin(ang)], axis=1)
    segs = [fl[i * seg_blobs:(i + 1) * seg_blobs] for i in range(n_seg)]
    hinge = [np.array([-(axes[0] + a), 0.0, 0.0]),
             np.array([-(axes[0] + a + 1.0), 0.0, 0.0])]
    joints = [0.5 * (segs[i][-1] + segs[i + 1][0]) for i in range(n_seg - 1)]
    return [head] + segs, hinge, joints


def bacteria_wall(seed, n_bact=1000, a=0.05, box=250.0, hmin=1.0, hmax=5.0,
                  motor_torque=1.0, eta=1.0, **tmpl_kw):
    """Bacteria lying parallel to a no-slip wall: seeded lateral positions in
    a square of side ``box``, heights in [hmin, hmax] and azimuths; a motor
    torque +-motor_torque about the helix axis on the head and the first
    flagellum segment.  Each body's tracking point is its blob centroid, so
    the head's is the head centre.  With the defaults: 17,000 bodies,
    360,000 blobs, 17,000 links.

    Placing the template at azimuth psi is a plain rotation of the plane
    about z; the body orientation is the matching quaternion
    [cos(psi/2), 0, 0, sin(psi/2)].
    """
    rng = np.random.default_rng(np.random.Philox(seed))
    bodies, hinge, seg_joints = bacterium_template(a=a, **tmpl_kw)
    centroids = [b.mean(axis=0) for b in bodies]
    nb = len(bodies)
    xy = rng.uniform(0.0, box, (n_bact, 2))
    hz = rng.uniform(hmin, hmax, n_bact)
    psi = rng.uniform(0.0, 2 * math.pi, n_bact)

    def place(v, c, s, origin):
        return np.stack([origin[0] + c * v[..., 0] - s * v[..., 1],
                         origin[1] + s * v[..., 0] + c * v[..., 1],
                         origin[2] + v[..., 2]], axis=-1)

    q, theta, rho, F, assembly = [], [], [], [], []
    body_p, body_q, joints = [], [], []
    offs = [0]
    for b in range(n_bact):
        c, s = math.cos(psi[b]), math.sin(psi[b])
        origin = np.array([xy[b, 0], xy[b, 1], hz[b]])
        base = len(q)
        for k in range(nb):
            q.append(place(centroids[k], c, s, origin))
            theta.append([math.cos(psi[b] / 2), 0.0, 0.0, math.sin(psi[b] / 2)])
            rho.append(bodies[k] - centroids[k])
            offs.append(offs[-1] + len(bodies[k]))
            assembly.append(b)
            f = np.zeros(6)
            axis = np.array([c, s, 0.0])
            if k == 0:
                f[3:] = motor_torque * axis
            elif k == 1:
                f[3:] = -motor_torque * axis
            F.append(f)
        for hpt in hinge:
            body_p.append(base); body_q.append(base + 1)
            joints.append(place(hpt, c, s, origin))
        for i, jp in enumerate(seg_joints):
            body_p.append(base + 1 + i); body_q.append(base + 2 + i)
            joints.append(place(jp, c, s, origin))
    return dict(name="bacteria_wall", eta=eta, a=a, wall=1,
                q=np.array(q), theta=np.array(theta),
                blob_offset=np.array(offs, dtype=np.int64),
                rho=np.concatenate(rho), F=np.array(F),
                assembly=np.array(assembly, dtype=np.int64),
                body_p=np.array(body_p, dtype=np.int64),
                body_q=np.array(body_q, dtype=np.int64),
                joints=np.array(joints), dl=None)


def _quat_axis_angle(axis, ang):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    return np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * axis])


def _quat_mul(q2, q1):
    s2, p2, s1, p1 = q2[0], q2[1:], q1[0], q1[1:]
    return np.concatenate([[s2 * s1 - p2 @ p1], s2 * p1 + s1 * p2 + np.cross(p2, p1)])


def _quat_rot(q):
    s, p = q[0], q[1:]
    return 2.0 * (np.outer(p, p) + s * np.array([[0, -p[2], p[1]], [p[2], 0, -p[0]], [-p[1], p[0], 0]])
                  + (s * s - 0.5) * np.eye(3))


def bacteria_periodic(seed, lattice=(10, 10, 10), spacing=(15.0, 3.0, 3.0), tilt=0.02, a=0.05,
                      motor_torque=1.0, eta=1.0, jitter=(0.02, 0.05, 0.05), **tmpl_kw):
    """Bacteria in a triply periodic box (the periodic suspensions of Sec.
    5.3, here without the wall): one bacterium per site of a lattice with
    the given spacing (box = lattice x spacing), its head centre jittered by
    up to ``jitter`` x spacing per axis, long axis along x tilted by up to
    ``tilt`` radians about a random perpendicular axis and spun by a random
    angle about itself: an aligned suspension.  With the defaults the bodies
    cannot overlap: a bacterium spans 13.5 along x and at most 0.55 + 0.24
    (head radius plus the tilt over its length) across, so neighbouring
    bacteria stay at least 0.95 apart along x and 1.1 across.
    Motor torques as in bacteria_wall.  With the defaults: 1,000 bacteria,
    360,000 blobs in a 150 x 30 x 30 box.  Returns the workload dict with
    ``box``."""
    rng = np.random.default_rng(np.random.Philox(seed))
    bodies, hinge, seg_joints = bacterium_template(a=a, **tmpl_kw)
    centroids = [b.mean(axis=0) for b in bodies]
    nb = len(bodies)
    box = np.array(lattice, dtype=np.float64) * np.array(spacing, dtype=np.float64)
    q, theta, rho, F, assembly = [], [], [], [], []
    body_p, body_q, joints = [], [], []
    offs = [0]
    b = 0
    for ix in range(lattice[0]):
        for iy in range(lattice[1]):
            for iz in range(lattice[2]):
                origin = (np.array([ix, iy, iz]) + 0.5 +
                          rng.uniform(-1.0, 1.0, 3) * np.asarray(jitter)) * np.array(spacing)
                spin = _quat_axis_angle([1.0, 0.0, 0.0], rng.uniform(0.0, 2 * math.pi))
                phi = rng.uniform(0.0, 2 * math.pi)
                tq = _quat_axis_angle([0.0, math.cos(phi), math.sin(phi)], rng.uniform(0.0, tilt))
                qq = _quat_mul(tq, spin)
                R = _quat_rot(qq)
                base = len(q)
                axis = R @ np.array([1.0, 0.0, 0.0])
                for k in range(nb):
                    q.append(origin + R @ centroids[k])
                    theta.append(qq.copy())
                    rho.append(bodies[k] - centroids[k])
                    offs.append(offs[-1] + len(bodies[k]))
                    assembly.append(b)
                    f = np.zeros(6)
                    if k == 0:
                        f[3:] = motor_torque * axis
                    elif k == 1:
                        f[3:] = -motor_torque * axis
                    F.append(f)
                for hpt in hinge:
                    body_p.append(base); body_q.append(base + 1)
                    joints.append(origin + R @ hpt)
                for i, jp in enumerate(seg_joints):
                    body_p.append(base + 1 + i); body_q.append(base + 2 + i)
                    joints.append(origin + R @ jp)
                b += 1
    return dict(name="bacteria_periodic", eta=eta, a=a, wall=0, box=box,
                q=np.array(q), theta=np.array(theta),
                blob_offset=np.array(offs, dtype=np.int64),
                rho=np.concatenate(rho), F=np.array(F),
                assembly=np.array(assembly, dtype=np.int64),
                body_p=np.array(body_p, dtype=np.int64),
                body_q=np.array(body_q, dtype=np.int64),
                joints=np.array(joints), dl=None)


def random_blobs(seed, n, box=None, a=0.1, wall=0, hmin=None, hmax=None):
    """Loose blobs for matvec tests: uniform in a cube whose side keeps the
    number density of ``n`` blobs moderate; above a wall the heights are
    uniform in [hmin, hmax].  Returns (positions (n, 3), forces (n, 3))."""
    rng = np.random.default_rng(np.random.Philox(seed))
    if box is None:
        box = max(1.0, (n / 8.0) ** (1.0 / 3.0))
    r = rng.uniform(0.0, box, (n, 3))
    if wall:
        lo = 2.0 * a if hmin is None else hmin
        hi = box if hmax is None else hmax
        r[:, 2] = rng.uniform(lo, hi, n)
    lam = rng.standard_normal((n, 3))
    return r, lam


def counts(w):
    """(blobs, bodies, links, unknowns) of a workload, unknowns ordered
    y = (lambda, U, phi) as in Eq. linear_system."""
    nb = int(w["blob_offset"][-1])
    M = len(w["q"])
    P = len(w["body_p"])
    return nb, M, P, 3 * nb + 6 * M + 3 * P
