"""Seeded rigid-aggregate suspensions.

Aggregates are grown by random sequential attachment: each new bead touches
(centre distance exactly 2a) a uniformly chosen existing bead in a uniform
random direction; a placement closer than 2a(1 - 1e-12) to any existing bead
of the same aggregate is rejected.  Aggregates are inserted into a periodic
cube with uniform centres and uniform random orientations (normalised 4-D
Gaussian quaternions); an insertion is rejected if any bead of another body
comes within a surface gap h_gen.  Bead volume fraction
phi = N_tot (4/3) pi a^3 / L^3.

Returned positions are unwrapped per aggregate (an aggregate is never split
across the box boundary); centres lie in [0, L).
"""

import math

import numpy as np

__all__ = [
    "random_attachment_aggregate",
    "doublet",
    "random_rotation",
    "pack_suspension",
    "box_for_phi",
    "suspension",
    "config_doublets",
    "config_aggregates",
    "random_forces",
    "compress_suspension",
    "compress_mixed",
    "mixed_suspension",
    "dense_suspension",
    "replicate_box",
    "batch_workload",
    "rod",
    "rod_suspension",
]


def random_attachment_aggregate(n_b, rng, a=1.0):
    """Bead offsets (n_b, 3) of one aggregate, centred on its bead centroid."""
    pts = [np.zeros(3)]
    while len(pts) < n_b:
        base = pts[rng.integers(len(pts))]
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        cand = base + 2.0 * a * d
        P = np.array(pts)
        if np.all(np.linalg.norm(P - cand, axis=1) >= 2.0 * a * (1.0 - 1e-12)):
            pts.append(cand)
    P = np.array(pts)
    return P - P.mean(axis=0)


def doublet(a=1.0):
    return np.array([[-a, 0.0, 0.0], [a, 0.0, 0.0]])


def random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def box_for_phi(n_tot, phi, a=1.0):
    return (n_tot * (4.0 / 3.0) * math.pi * a ** 3 / phi) ** (1.0 / 3.0)


class _Hash:
    """Uniform cell hash over the periodic box for overlap rejection."""

    def __init__(self, L, cell):
        self.L = L
        self.n = max(1, int(L // cell))
        self.cell = L / self.n
        self.cells = {}

    def key(self, p):
        c = np.floor((p % self.L) / self.cell).astype(int) % self.n
        return tuple(c)

    def near(self, p):
        c = self.key(p)
        n = self.n
        rng = (-1, 0, 1) if n >= 3 else tuple(range(n))
        out = []
        seen = set()
        for dx in rng:
            for dy in rng:
                for dz in rng:
                    k = ((c[0] + dx) % n, (c[1] + dy) % n, (c[2] + dz) % n)
                    if k in seen:
                        continue
                    seen.add(k)
                    out.extend(self.cells.get(k, ()))
        return out

    def add(self, p, idx):
        self.cells.setdefault(self.key(p), []).append(idx)


def pack_suspension(shapes, L, rng, a=1.0, h_gen=0.1, max_tries=20000):
    """Insert rigid shapes (list of (n_b,3) offset arrays) into a cube of side L.

    Returns pos (N_tot, 3), body (N_tot,) int32."""
    contact = 2.0 * a + h_gen
    hsh = _Hash(L, contact)
    allpos = []
    body = []
    for J, shp in enumerate(shapes):
        for _ in range(max_tries):
            R = random_rotation(rng)
            c = rng.uniform(0.0, L, size=3)
            P = c + shp @ R.T
            ok = True
            for p in P:
                for j in hsh.near(p):
                    d = allpos[j] - p
                    d -= L * np.round(d / L)
                    if d @ d < contact * contact:
                        ok = False
                        break
                if not ok:
                    break
            if ok:
                break
        else:
            raise RuntimeError("suspension packing jammed at body %d" % J)
        for p in P:
            hsh.add(p, len(allpos))
            allpos.append(p)
            body.append(J)
    return np.array(allpos), np.array(body, dtype=np.int32)


def suspension(n_agg, n_b, phi, seed, a=1.0, h_gen=0.1):
    """n_agg random-attachment aggregates of n_b beads at bead volume fraction
    phi.  Up to phi = 0.12 by random sequential insertion alone; denser
    suspensions are compressed from phi = 0.12 (compress_suspension)."""
    rng = np.random.default_rng(seed)
    shapes = [random_attachment_aggregate(n_b, rng, a) for _ in range(n_agg)]
    if phi > 0.12:
        return compress_suspension(np.array(shapes), phi, seed + 1, a, h_gen)
    L = box_for_phi(n_agg * n_b, phi, a)
    pos, body = pack_suspension(shapes, L, rng, a, h_gen)
    return pos, body, L


def rod(n_b, a=1.0):
    """A straight rigid rod of n_b touching beads (centre spacing 2a) along x,
    centred on its bead centroid."""
    x = (np.arange(n_b) - 0.5 * (n_b - 1)) * 2.0 * a
    return np.stack([x, np.zeros(n_b), np.zeros(n_b)], axis=1)


def rod_suspension(n_rods, n_b, phi, seed, a=1.0, h_gen=0.1):
    """n_rods straight n_b-bead rods at bead volume fraction phi, uniform
    centres and orientations, no inter-rod gap below h_gen (the rod workload
    of the scaling study, Sec. 3.3).  A rod must be shorter than half the
    box (it would otherwise reach its own periodic image)."""
    rng = np.random.default_rng(seed)
    L = box_for_phi(n_rods * n_b, phi, a)
    if 2.0 * a * n_b >= 0.5 * L:
        raise ValueError("rod of %d beads does not fit half of the box L = %.1f" % (n_b, L))
    # random sequential insertion of long rods saturates early (27-bead rods
    # jam near phi 0.1): above phi0 = 1.5 / n_b insert at phi0 and compress
    phi0 = 1.5 / n_b
    if phi > phi0:
        return compress_suspension(np.array([rod(n_b, a)] * n_rods), phi, seed + 1, a, h_gen, phi0=phi0)
    pos, body = pack_suspension([rod(n_b, a)] * n_rods, L, rng, a, h_gen, max_tries=200000)
    return pos, body, L


def config_doublets(n_agg=16, L=40.0, seed=1, a=1.0):
    """Rigid touching doublets (centre separation 2a) at uniform centres and
    uniform random orientations in a cube of side L."""
    rng = np.random.default_rng(seed)
    shapes = [doublet(a) for _ in range(n_agg)]
    pos, body = pack_suspension(shapes, L, rng, a, h_gen=0.1)
    return pos, body, L


def config_aggregates(n_agg, n_b, phi, seed=1, a=1.0):
    return suspension(n_agg, n_b, phi, seed, a)


def random_forces(n_agg, seed, scale=1.0):
    """Seeded aggregate forces / torques (n_agg, 6), standard normal x scale."""
    rng = np.random.default_rng(seed + 7919)
    return scale * rng.normal(size=(n_agg, 6))


# ---------------------------------------------------------------------------
# dense packings: random sequential insertion at a looser density, then
# affine compression of the centres with overlap-removing Monte Carlo moves
# ---------------------------------------------------------------------------


def _rot_from_quat(q):
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _overlap_mask(P, body, L, contact, nbody):
    """Bodies having any bead of another body closer than `contact`
    (minimum image).  P (Nt, 3)."""
    n = max(1, int(L // contact))
    cs = L / n
    c = np.floor((P % L) / cs).astype(np.int64) % n
    cid = (c[:, 0] * n + c[:, 1]) * n + c[:, 2]
    order = np.argsort(cid, kind="stable")
    cnt = np.bincount(cid, minlength=n ** 3)
    m = int(cnt.max())
    table = -np.ones((n ** 3, m), dtype=np.int64)
    start = np.concatenate([[0], np.cumsum(cnt)[:-1]])
    sc = cid[order]
    slot = np.arange(len(order)) - start[sc]
    table[sc, slot] = order
    bad = np.zeros(nbody, dtype=bool)
    offs = (-1, 0, 1) if n >= 3 else tuple(range(n))
    seen = set()
    for dx in offs:
        for dy in offs:
            for dz in offs:
                key = (dx % n, dy % n, dz % n)
                if key in seen:
                    continue
                seen.add(key)
                nc = (((c[:, 0] + dx) % n) * n + (c[:, 1] + dy) % n) * n + (c[:, 2] + dz) % n
                J = table[nc]  # (Nt, m)
                valid = J >= 0
                Jc = np.where(valid, J, 0)
                d = P[Jc] - P[:, None, :]
                d -= L * np.round(d / L)
                r2 = np.einsum("nmk,nmk->nm", d, d)
                hit = valid & (r2 < contact * contact) & (body[Jc] != body[:, None])
                bad[body[hit.any(axis=1)]] = True
    return bad


def _close_pairs(P, body, L, contact):
    """Inter-body bead pairs (i < j) closer than `contact` (minimum image):
    returns i, j, d = P[j] - P[i] (minimum image)."""
    from scipy.spatial import cKDTree

    W = np.mod(P, L)
    W[W >= L] = 0.0
    pr = cKDTree(W, boxsize=L).query_pairs(contact, output_type="ndarray")
    if len(pr) == 0:
        z = np.zeros(0, dtype=np.int64)
        return z, z, np.zeros((0, 3))
    i, j = pr[:, 0], pr[:, 1]
    keep = body[i] != body[j]
    i, j = i[keep], j[keep]
    d = P[j] - P[i]
    d -= L * np.round(d / L)
    return i, j, d


def compress_suspension(shapes, phi, seed, a=1.0, h_gen=0.1, phi0=0.12,
                        step=0.99, max_iter=4000):
    """Pack equal-size rigid shapes at bead volume fraction phi.

    Random sequential insertion at phi0, then repeated affine compression of
    the body centres (factor `step` in L), each followed by a soft-repulsion
    relaxation: every inter-body bead pair closer than 2a + h_gen pushes its
    two bodies apart (rigid translation and rotation driven by the summed
    pair forces and torques) until no such pair is left."""
    rng = np.random.default_rng(seed)
    N, nb_ = shapes.shape[0], shapes.shape[1]
    Lt = box_for_phi(N * nb_, phi, a)
    L = box_for_phi(N * nb_, min(phi0, phi), a)
    pos, body = pack_suspension(list(shapes), L, rng, a, h_gen)
    target = 2.0 * a + 1.01 * h_gen  # pairs closer than this are pushed ...
    push = 2.0 * a + 1.25 * h_gen    # ... towards this separation
    contact = 2.0 * a + h_gen
    P = pos.reshape(N, nb_, 3)
    C = P.mean(axis=1)
    off = P - C[:, None, :]
    bodyidx = np.repeat(np.arange(N), nb_)

    def beads():
        return (C[:, None, :] + off).reshape(-1, 3)

    def rotate(off_, w):
        th = np.linalg.norm(w, axis=1)
        k = np.where(th[:, None] > 0, w / np.maximum(th, 1e-300)[:, None], 0.0)
        ct, st = np.cos(th)[:, None, None], np.sin(th)[:, None, None]
        kx = np.einsum("nj,nbj->nb", k, off_)[..., None]
        cr = np.cross(k[:, None, :], off_)
        return off_ * ct + cr * st + k[:, None, :] * kx * (1 - ct)

    while True:
        for _ in range(max_iter):
            Pb = beads()
            i, j, d = _close_pairs(Pb, bodyidx, L, target)
            if len(i) == 0:
                break
            r = np.linalg.norm(d, axis=1)
            f = ((push - r) / np.maximum(r, 1e-12))[:, None] * d  # push j away from i
            F = np.zeros((N, 3))
            T = np.zeros((N, 3))
            np.add.at(F, bodyidx[j], 0.5 * f)
            np.add.at(F, bodyidx[i], -0.5 * f)
            oi = off.reshape(-1, 3)[i]
            oj = off.reshape(-1, 3)[j]
            np.add.at(T, bodyidx[j], np.cross(oj, 0.5 * f))
            np.add.at(T, bodyidx[i], np.cross(oi, -0.5 * f))
            C = (C + 0.6 * F) % L
            off = rotate(off, 0.6 * T / (np.einsum("nbk,nbk->n", off, off)[:, None] + a * a))
        else:
            raise RuntimeError("relaxation stalled at L=%.3f" % L)
        if L <= Lt * (1 + 1e-12):
            break
        Ln = max(L * step, Lt)
        C = C * (Ln / L)
        L = Ln
    Pb = beads()
    assert len(_close_pairs(Pb, bodyidx, L, contact)[0]) == 0
    return Pb, bodyidx.astype(np.int32), L


# ---------------------------------------------------------------------------
# batched form: independent suspensions of uneven bead and aggregate counts
# ---------------------------------------------------------------------------


def compress_mixed(shapes, phi, seed, a=1.0, h_gen=0.1, phi0=0.12, step=0.98, max_iter=400):
    """compress_suspension for shapes of different bead counts (a list of
    (n_b, 3) offset arrays): random sequential insertion at phi0, then affine
    compression of the body centres with soft-repulsion relaxation.  Large
    branched aggregates can jam below the requested phi; the densest packing
    reached is then returned (its box L gives the actual phi)."""
    rng = np.random.default_rng(seed)
    N = len(shapes)
    nbs = np.array([len(s_) for s_ in shapes])
    Nt = int(nbs.sum())
    Lt = box_for_phi(Nt, phi, a)
    # large bodies first; a looser start when insertion jams
    phi_start = min(phi0, phi)
    while True:
        L = box_for_phi(Nt, phi_start, a)
        try:
            pos, body = pack_suspension(list(shapes), L, rng, a, h_gen)
            break
        except RuntimeError:
            phi_start *= 0.7
    body = body.astype(np.int64)
    target = 2.0 * a + 1.01 * h_gen
    push = 2.0 * a + 1.25 * h_gen
    contact = 2.0 * a + h_gen
    C = np.zeros((N, 3))
    np.add.at(C, body, pos)
    C /= nbs[:, None]
    off = pos - C[body]
    inertia = np.zeros(N)
    np.add.at(inertia, body, np.einsum("nk,nk->n", off, off))

    def rotate(off_, w):
        wb = w[body]
        th = np.linalg.norm(wb, axis=1)
        k = np.where(th[:, None] > 0, wb / np.maximum(th, 1e-300)[:, None], 0.0)
        ct, st = np.cos(th)[:, None], np.sin(th)[:, None]
        kx = np.einsum("nj,nj->n", k, off_)[:, None]
        return off_ * ct + np.cross(k, off_) * st + k * kx * (1 - ct)

    def relax(C, off):
        for _ in range(max_iter):
            Pb = C[body] + off
            i, j, d = _close_pairs(Pb, body, L, target)
            if len(i) == 0:
                return C, off, True
            r = np.linalg.norm(d, axis=1)
            f = ((push - r) / np.maximum(r, 1e-12))[:, None] * d
            F = np.zeros((N, 3))
            T = np.zeros((N, 3))
            np.add.at(F, body[j], 0.5 * f)
            np.add.at(F, body[i], -0.5 * f)
            np.add.at(T, body[j], np.cross(off[j], 0.5 * f))
            np.add.at(T, body[i], np.cross(off[i], -0.5 * f))
            C = (C + 0.6 * F / np.sqrt(nbs)[:, None]) % L
            off = rotate(off, 0.6 * T / (inertia[:, None] + a * a))
        return C, off, False

    # a compression whose relaxation stalls is undone and retried with half
    # the strain
    C, off, ok = relax(C, off)
    if not ok:
        raise RuntimeError("relaxation stalled at L=%.3f" % L)
    while L > Lt * (1 + 1e-12):
        Ln = max(L * step, Lt)
        C0, off0, L0 = C.copy(), off.copy(), L
        C = C * (Ln / L)
        L = Ln
        C, off, ok = relax(C, off)
        if not ok:
            C, off, L = C0, off0, L0
            step = 1.0 - 0.5 * (1.0 - step)
            if step > 1.0 - 1e-3:
                break  # jammed: keep the densest packing reached
    Pb = C[body] + off
    assert len(_close_pairs(Pb, body, L, contact)[0]) == 0
    return Pb, body.astype(np.int32), L


def _extent(shape):
    d = shape[:, None, :] - shape[None, :, :]
    return float(np.sqrt((d * d).sum(-1).max())) if len(shape) > 1 else 0.0


def mixed_suspension(n_beads, phi, seed, size_lo=2, size_hi=64, a=1.0, h_gen=0.1):
    """n_beads beads in random-attachment aggregates whose sizes are drawn
    uniformly from size_lo..size_hi, at bead volume fraction phi.

    The last aggregate is trimmed so the total is exactly n_beads (a trimmed
    remainder below size_lo joins the previous aggregate).  An aggregate
    whose extent (largest bead-centre distance + 2a) exceeds half the box is
    regrown at half its size: a body larger than that would touch its own
    periodic images."""
    rng = np.random.default_rng(seed)
    L = box_for_phi(n_beads, phi, a)
    sizes = []
    while sum(sizes) < n_beads:
        sizes.append(int(rng.integers(size_lo, size_hi + 1)))
    sizes[-1] -= sum(sizes) - n_beads
    if sizes[-1] < size_lo and len(sizes) > 1:
        sizes[-2] += sizes.pop()
    shapes = []
    for nb in sizes:
        parts = [nb]
        out = []
        while parts:
            k = parts.pop()
            shp = random_attachment_aggregate(k, rng, a)
            if k >= 2 * size_lo and _extent(shp) + 2 * a > 0.5 * L:
                parts += [k // 2, k - k // 2]
            else:
                out.append(shp)
        shapes += out
    shapes.sort(key=len, reverse=True)  # insert large bodies first
    if phi > 0.12:
        return compress_mixed(shapes, phi, seed + 1, a, h_gen)
    pos, body = pack_suspension(shapes, L, rng, a, h_gen)
    return pos, body, L


def dense_suspension(n_agg, n_b, phi, seed, a=1.0, h_gen=0.1):
    """n_agg random-attachment aggregates of n_b beads at bead volume
    fraction phi, compressed like the batched form's systems: where the
    branched aggregates jam before phi (16-bead aggregates near phi = 0.3),
    the densest packing reached is kept and its box L gives the actual
    phi.  Returns (bead_pos, agg_id, L)."""
    rng = np.random.default_rng(seed)
    shapes = [random_attachment_aggregate(n_b, rng, a) for _ in range(n_agg)]
    if phi <= 0.12:
        L = box_for_phi(n_agg * n_b, phi, a)
        pos, body = pack_suspension(shapes, L, rng, a, h_gen)
        return pos, body, L
    return compress_mixed(shapes, phi, seed + 1, a, h_gen)


def replicate_box(pos, body, L, reps):
    """Periodic replica of a cubic suspension: the box of side L tiled
    reps = (rx, ry, rz) times (the larger box is a non-cubic periodic cell
    when the reps differ).  Returns (bead_pos, agg_id, box sides); the copy
    (i, j, k) is shifted by (i, j, k) L and its aggregate ids offset by the
    number of aggregates before it.  A periodic suspension and its tiling are
    the same infinite suspension, at the same volume fraction."""
    pos = np.asarray(pos, dtype=np.float64)
    body = np.asarray(body)
    nb = int(body.max()) + 1
    out_p, out_b = [], []
    c = 0
    for i in range(reps[0]):
        for j in range(reps[1]):
            for k in range(reps[2]):
                out_p.append(pos + L * np.array([i, j, k], dtype=np.float64))
                out_b.append(body + c * nb)
                c += 1
    return (np.concatenate(out_p), np.concatenate(out_b).astype(np.int32),
            (L * reps[0], L * reps[1], L * reps[2]))


def batch_workload(n_sys, seed, n_lo=256, n_hi=8192, phi_lo=0.05, phi_hi=0.3, size_lo=2,
                   size_hi=64):
    """Independent suspensions: bead counts round(exp(U[ln n_lo, ln n_hi])),
    volume fractions U[phi_lo, phi_hi], aggregate sizes U{size_lo..size_hi}.
    Returns a list of (bead_pos, agg_id, L, phi), phi the volume fraction
    reached (below the drawn one where the aggregates jammed first)."""
    rng = np.random.default_rng(seed)
    n = np.rint(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=n_sys))).astype(int)
    phi = rng.uniform(phi_lo, phi_hi, size=n_sys)
    out = []
    for s in range(n_sys):
        pos, body, L = mixed_suspension(int(n[s]), float(phi[s]), seed * 1000 + s, size_lo, size_hi)
        out.append((pos, body, L, len(pos) * 4.0 / 3.0 * math.pi / L ** 3))
    return out
