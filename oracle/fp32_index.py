"""Index mode of the oracle: every integer-deciding quantity in IEEE float32.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper leaves the rasterizer's arithmetic to the base 3DGS method (Supp.
"Implementation Details") and asks for a tile mask and per-tile depth order
built from the projection (Supp. "Local Optimization Kernel", item 1). Which
tiles a Gaussian touches, the bits of its depth key, and whether a Gaussian's
centre lands in a change mask (Sec. 3.2, Supp. majority-voting equation) are
integer results decided by floating point. To compare them bit for bit, this
module fixes one float32 operation sequence: every +, -, *, / and sqrt is a
single correctly rounded float32 operation (NumPy evaluates each ufunc call
separately, so nothing is fused), floor/ceil/rint are exact, and exp is the
Cody-Waite reduction plus a degree-7 Taylor polynomial written out below, so
that no vendor math routine decides an integer.

Readings of points the paper leaves silent:
  * pinhole camera, pixel (i, j) covers [i, i+1) x [j, j+1);
  * near plane z > znear (0.2), otherwise culled / counted outside the image;
  * 2D covariance gets +0.3 on the diagonal; the perspective Jacobian uses the
    tangent clamped to 1.3x the half field of view;
  * radius r = ceil(3 sqrt(lambda_max)), lambda_max = m + sqrt(max(0.1, m^2 -
    det)), m = (a + c) / 2;
  * tile rectangle: tiles [floor((u - r)/16), floor((u + r)/16)] clamped to the
    grid, same for v; empty if lo > hi;
  * key = (global tile id << 32) | float bits of the camera-space depth,
    pairs emitted per view in Gaussian order then row-major tile order, then a
    stable sort: equal depths keep the lower Gaussian index first.
"""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np

F = np.float32
TILE = 16


def f32(x) -> np.ndarray:
    return np.asarray(x, dtype=np.float32)


# ---------------------------------------------------------------------------
# exp in float32: Cody & Waite argument reduction (ln 2 split in a high part
# with 12 trailing zero bits and a low part), then e^r by the Taylor series to
# degree 7 on |r| <= ln(2)/2, evaluated by Horner's rule one rounded operation
# at a time, then scaled by 2^k built from its exponent bits.

_LOG2E = F(1.4426950408889634)
_LN2 = 0.6931471805599453
_LN2_HI = np.frombuffer(
    (np.frombuffer(F(_LN2).tobytes(), np.uint32) & np.uint32(0xFFFFF000)).tobytes(),
    np.float32)[0]
_LN2_LO = F(_LN2 - float(_LN2_HI))
_TAYLOR = [F(1.0 / f) for f in (5040.0, 720.0, 120.0, 24.0, 6.0, 2.0, 1.0, 1.0)]
EXP_LO, EXP_HI = F(-87.0), F(88.0)


def exp32(x) -> np.ndarray:
    x = np.minimum(np.maximum(f32(x), EXP_LO), EXP_HI)
    kf = np.rint(x * _LOG2E).astype(np.float32)
    r = (x - kf * _LN2_HI) - kf * _LN2_LO
    p = np.full_like(r, _TAYLOR[0])
    for c in _TAYLOR[1:]:
        p = p * r + c
    k = kf.astype(np.int32)
    two_k = ((k + 127).astype(np.uint32) << np.uint32(23)).view(np.float32)
    return (p * two_k).astype(np.float32)


# ---------------------------------------------------------------------------
# camera and parameter canonicalisation: the library receives float32.

def camera32(cam) -> Dict[str, object]:
    return {
        "R": f32(np.asarray(cam["R"]).reshape(9)),
        "t": f32(cam["t"]),
        "pos": f32(cam["pos"]),
        "fx": F(cam["fx"]), "fy": F(cam["fy"]),
        "cx": F(cam["cx"]), "cy": F(cam["cy"]),
        "znear": F(cam["znear"]),
        "W": int(cam["width"]), "H": int(cam["height"]),
    }


def tiles_of(cam) -> tuple:
    W, H = int(cam["width"]), int(cam["height"])
    return (W + TILE - 1) // TILE, (H + TILE - 1) // TILE


def camera_space(means: np.ndarray, c: Dict[str, object]):
    """p = R mu + t, each row summed left to right then t added."""
    R, t = c["R"], c["t"]
    x, y, z = f32(means[:, 0]), f32(means[:, 1]), f32(means[:, 2])
    px = ((R[0] * x + R[1] * y) + R[2] * z) + t[0]
    py = ((R[3] * x + R[4] * y) + R[5] * z) + t[1]
    pz = ((R[6] * x + R[7] * y) + R[8] * z) + t[2]
    return px, py, pz


def centre_pixel(px, py, pz, c):
    """Image coordinates of a camera-space point: u = fx (x/z) + cx."""
    xz = px / pz
    yz = py / pz
    u = c["fx"] * xz + c["cx"]
    v = c["fy"] * yz + c["cy"]
    return xz, yz, u, v


# ---------------------------------------------------------------------------
# Change-mask lifting (Sec. 3.2 "Mask Majority Voting"; Supp. "Identifying
# Changed 3D Regions via Majority Voting", the voting equation).

def votes(means: np.ndarray, cams: Sequence, masks: Sequence[np.ndarray]):
    """Per Gaussian: c = number of views whose change mask holds the projected
    centre, o = number of views where the centre falls outside the image (or
    behind the near plane). A centre inside the image on a 0 pixel counts in
    neither."""
    n = means.shape[0]
    c_cnt = np.zeros(n, np.int32)
    o_cnt = np.zeros(n, np.int32)
    for cam, mask in zip(cams, masks):
        c = camera32(cam)
        px, py, pz = camera_space(means, c)
        front = pz > c["znear"]
        with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
            _, _, u, v = centre_pixel(px, py, pz, c)
        inside = front & (u >= F(0)) & (u < F(c["W"])) & (v >= F(0)) & (v < F(c["H"]))
        iu = np.where(inside, np.floor(np.where(inside, u, 0)), 0).astype(np.int64)
        iv = np.where(inside, np.floor(np.where(inside, v, 0)), 0).astype(np.int64)
        hit = inside & (mask[iv, iu] != 0)
        c_cnt += hit
        o_cnt += ~inside
    return c_cnt, o_cnt


def vote_rule(c: np.ndarray, o: np.ndarray, n_views: int, mode: int = 0) -> np.ndarray:
    """mode 0: g in O^t iff (4/3) o < |I^t| < 2 c, evaluated in integers as
    4 o < 3 V and V < 2 c. mode 1 ("All Vote", Table 4 (b)): c == V."""
    c = np.asarray(c, np.int64)
    o = np.asarray(o, np.int64)
    if mode == 1:
        return c == n_views
    return (4 * o < 3 * n_views) & (n_views < 2 * c)


# ---------------------------------------------------------------------------
# Projection decisions (base 3DGS EWA projection, restated).

def project_index(scene: Dict[str, np.ndarray], cam) -> Dict[str, np.ndarray]:
    """float32 projection of every Gaussian for one camera.

    Returns valid (bool), u, v, z (float32), radius (float32, integer valued),
    the tile rectangle (ints, inclusive) and the depth-key bits."""
    c = camera32(cam)
    Tx, Ty = tiles_of(cam)
    means = f32(scene["means"])
    with np.errstate(all="ignore"):
        px, py, pz = camera_space(means, c)
        valid = pz > c["znear"]
        xz, yz, u, v = centre_pixel(px, py, pz, c)

        s = exp32(scene["log_scales"])
        s0, s1, s2 = s[:, 0], s[:, 1], s[:, 2]
        q = f32(scene["quats"])
        qw, qx, qy, qz = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
        n2 = ((qw * qw + qx * qx) + qy * qy) + qz * qz
        valid &= n2 > F(0)
        nrm = np.sqrt(n2)
        w, x, y, z = qw / nrm, qx / nrm, qy / nrm, qz / nrm
        xx, yy, zz = x * x, y * y, z * z
        xy, xzq, yzq = x * y, x * z, y * z
        wx, wy, wz = w * x, w * y, w * z
        one, two = F(1), F(2)
        r00 = one - two * (yy + zz); r01 = two * (xy - wz); r02 = two * (xzq + wy)
        r10 = two * (xy + wz); r11 = one - two * (xx + zz); r12 = two * (yzq - wx)
        r20 = two * (xzq - wy); r21 = two * (yzq + wx); r22 = one - two * (xx + yy)
        M = [[r00 * s0, r01 * s1, r02 * s2],
             [r10 * s0, r11 * s1, r12 * s2],
             [r20 * s0, r21 * s1, r22 * s2]]

        def dot3(a, b):
            return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]

        S00 = dot3(M[0], M[0]); S01 = dot3(M[0], M[1]); S02 = dot3(M[0], M[2])
        S11 = dot3(M[1], M[1]); S12 = dot3(M[1], M[2]); S22 = dot3(M[2], M[2])
        S = [[S00, S01, S02], [S01, S11, S12], [S02, S12, S22]]

        half = F(0.5)
        limx = F(1.3) * ((half * F(c["W"])) / c["fx"])
        limy = F(1.3) * ((half * F(c["H"])) / c["fy"])
        txz = np.minimum(np.maximum(xz, -limx), limx)
        tyz = np.minimum(np.maximum(yz, -limy), limy)
        tx = txz * pz
        ty = tyz * pz
        z2 = pz * pz
        J00 = c["fx"] / pz
        J02 = -((c["fx"] * tx) / z2)
        J11 = c["fy"] / pz
        J12 = -((c["fy"] * ty) / z2)
        R = c["R"]
        T0 = [J00 * R[0] + J02 * R[6], J00 * R[1] + J02 * R[7], J00 * R[2] + J02 * R[8]]
        T1 = [J11 * R[3] + J12 * R[6], J11 * R[4] + J12 * R[7], J11 * R[5] + J12 * R[8]]
        U0 = [dot3(T0, [S[0][j], S[1][j], S[2][j]]) for j in range(3)]
        U1 = [dot3(T1, [S[0][j], S[1][j], S[2][j]]) for j in range(3)]
        dil = F(0.3)
        a = dot3(U0, T0) + dil
        b = dot3(U0, T1)
        cc = dot3(U1, T1) + dil
        det = a * cc - b * b
        valid &= det > F(0)
        mid = half * (a + cc)
        disc = mid * mid - det
        lam = mid + np.sqrt(np.maximum(F(0.1), disc))
        radius = np.ceil(F(3) * np.sqrt(lam))
        valid &= (u == u) & (v == v) & (radius == radius)

        ft = F(TILE)
        x0 = np.floor((u - radius) / ft)
        x1 = np.floor((u + radius) / ft)
        y0 = np.floor((v - radius) / ft)
        y1 = np.floor((v + radius) / ft)
        txl = np.maximum(x0, F(0)); txh = np.minimum(x1, F(Tx - 1))
        tyl = np.maximum(y0, F(0)); tyh = np.minimum(y1, F(Ty - 1))
        valid &= (txl <= txh) & (tyl <= tyh)

    def to_int(a):
        return np.where(valid, a, 0).astype(np.int64)

    return {
        "valid": valid,
        "u": u.astype(np.float32), "v": v.astype(np.float32),
        "z": pz.astype(np.float32), "radius": radius.astype(np.float32),
        "tx0": to_int(txl), "tx1": to_int(txh), "ty0": to_int(tyl), "ty1": to_int(tyh),
        "zbits": np.where(valid, pz, F(0)).astype(np.float32).view(np.uint32),
        "scales": s,
    }


# ---------------------------------------------------------------------------
# Tile mask (Supp. "Local Optimization Kernel", item 1): a tile is active iff
# the rectangle of at least one non-culled active Gaussian contains it.

def tile_mask(proj: Dict[str, np.ndarray], active: np.ndarray, cam) -> np.ndarray:
    Tx, Ty = tiles_of(cam)
    m = np.zeros((Ty, Tx), np.uint8)
    for g in np.flatnonzero(proj["valid"] & active):
        m[proj["ty0"][g]:proj["ty1"][g] + 1, proj["tx0"][g]:proj["tx1"][g] + 1] = 1
    return m


def batch_layout(cams: Sequence, n_gauss: int):
    """Global tile ids and record ids of a batch of views of one scene: view j's
    tiles start at the sum of earlier views' tile counts, its records at j*n."""
    tile_base, t = [], 0
    for cam in cams:
        tile_base.append(t)
        Tx, Ty = tiles_of(cam)
        t += Tx * Ty
    rec_base = [j * n_gauss for j in range(len(cams))]
    return tile_base, rec_base, t


def pairs(projs: List[Dict[str, np.ndarray]], masks: List[np.ndarray], cams: Sequence,
          n_gauss: int):
    """Emit (key, value) for every (Gaussian, active tile) pair, in view order,
    then Gaussian order, then row-major tile order (vectorised enumeration)."""
    tile_base, rec_base, n_tiles = batch_layout(cams, n_gauss)
    keys_all, vals_all = [], []
    for j, (p, m, cam) in enumerate(zip(projs, masks, cams)):
        Tx, Ty = tiles_of(cam)
        g = np.flatnonzero(p["valid"])
        if g.size == 0 or not m.any():
            continue
        # clip every rectangle to the bounding box of active tiles first
        ys, xs = np.nonzero(m)
        bx0, bx1, by0, by1 = xs.min(), xs.max(), ys.min(), ys.max()
        x0 = np.maximum(p["tx0"][g], bx0); x1 = np.minimum(p["tx1"][g], bx1)
        y0 = np.maximum(p["ty0"][g], by0); y1 = np.minimum(p["ty1"][g], by1)
        keep = (x0 <= x1) & (y0 <= y1)
        g, x0, x1, y0, y1 = g[keep], x0[keep], x1[keep], y0[keep], y1[keep]
        wdt = x1 - x0 + 1
        area = wdt * (y1 - y0 + 1)
        gi = np.repeat(np.arange(g.size), area)
        start = np.repeat(np.cumsum(area) - area, area)
        k = np.arange(gi.size) - start
        ty = y0[gi] + k // wdt[gi]
        tx = x0[gi] + k % wdt[gi]
        on = m[ty, tx] != 0
        gi, tx, ty = gi[on], tx[on], ty[on]
        tile = (tile_base[j] + ty * Tx + tx).astype(np.uint64)
        keys_all.append((tile << np.uint64(32)) | p["zbits"][g[gi]].astype(np.uint64))
        vals_all.append((rec_base[j] + g[gi]).astype(np.uint32))
    if not keys_all:
        return np.zeros(0, np.uint64), np.zeros(0, np.uint32), n_tiles
    return np.concatenate(keys_all), np.concatenate(vals_all), n_tiles


def sort_pairs(keys: np.ndarray, vals: np.ndarray):
    """Stable sort by key (equal keys keep emission order)."""
    order = np.argsort(keys, kind="stable")
    return keys[order], vals[order]


def tile_ranges(sorted_keys: np.ndarray, n_tiles: int) -> np.ndarray:
    """[start, end) of each global tile id in the sorted key array."""
    tiles = (sorted_keys >> np.uint64(32)).astype(np.int64)
    rng = np.zeros((n_tiles, 2), np.int64)
    if tiles.size:
        starts = np.searchsorted(tiles, np.arange(n_tiles), side="left")
        ends = np.searchsorted(tiles, np.arange(n_tiles), side="right")
        rng[:, 0] = np.where(ends > starts, starts, 0)
        rng[:, 1] = np.where(ends > starts, ends, 0)
    return rng


def key_bits(n_tiles: int) -> int:
    """Bits a key can use: 32 depth bits plus enough for the largest tile id."""
    return 32 + max(1, int(n_tiles - 1).bit_length())
