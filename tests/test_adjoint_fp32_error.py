"""Float32 error of the two ways to get the colour behind a list entry in a
front-to-back compositing adjoint (no GPU): as the final colour minus what has
been composited up to the entry (the library's backward pass: no division,
nothing stored per entry), or summed from the back. Both are emulated in
float32 against float64 for dL/dalpha of every (pixel, entry) of tiles of the
local workload; the first carries an error relative to the pixel colour, the
second relative to the colour behind, which is why the parity floor of the
GPU's gradients sits above that of a float32 evaluation of the oracle."""
import math

import numpy as np

from oracle import fp32_index as fx
from oracle import step as ostep
from oracle.projection import project, scene64
from paper_2506_21117_gb300 import synthetic as S

F = np.float32


def _pixel_errors(ids, u, v, con, op, rgb, px, py, g):
    T, al, Ts, used = 1.0, [], [], []
    for i in ids:  # float64 walk: the composited entries, alpha and T in front
        dx, dy = px + 0.5 - u[i], py + 0.5 - v[i]
        pw = -0.5 * (con[i, 0] * dx * dx + con[i, 2] * dy * dy) - con[i, 1] * dx * dy
        if pw > 0:
            continue
        a = min(0.99, op[i] * math.exp(pw))
        if a < 1 / 255:
            continue
        if T * (1 - a) < 1e-4:
            break
        al.append(a), Ts.append(T), used.append(i)
        T *= 1 - a
    n = len(used)
    behind = np.zeros((n, 3))
    acc = np.zeros(3)
    for k in range(n - 1, -1, -1):
        behind[k] = acc
        acc = acc + rgb[used[k]] * al[k] * Ts[k]
    exact = np.array([Ts[k] * (rgb[used[k]] @ g) - (behind[k] @ g) / (1 - al[k])
                      for k in range(n)])
    a32 = [F(a) for a in al]
    c32 = [rgb[i].astype(F) for i in used]
    g32 = g.astype(F)
    T32, C32, Ts32 = F(1), np.zeros(3, F), []
    for k in range(n):  # float32 forward: final colour and T in front of each entry
        Ts32.append(T32)
        C32 = (C32 + c32[k] * F(a32[k] * T32)).astype(F)
        T32 = F(T32 * (F(1) - a32[k]))
    R, sub = C32.copy(), []
    for k in range(n):  # final minus composited
        R = (R - c32[k] * F(a32[k] * Ts32[k])).astype(F)
        sub.append(F(Ts32[k] * F(c32[k] @ g32)) - F(F(g32 @ R) / (F(1) - a32[k])))
    acc32, back = np.zeros(3, F), [0.0] * n
    for k in range(n - 1, -1, -1):  # summed from the back
        back[k] = F(Ts32[k] * F(c32[k] @ g32)) - F(F(g32 @ acc32) / (F(1) - a32[k]))
        acc32 = (acc32 + c32[k] * F(a32[k] * Ts32[k])).astype(F)
    return (np.abs(np.array(sub, np.float64) - exact), np.abs(np.array(back, np.float64) - exact))


def test_colour_behind_by_subtraction_costs_accuracy():
    scene = S.uniform_scene(6000, 3, 5)
    cam = S.ring_cameras(3, 4.0, 100, 75)[0]
    pidx = fx.project_index(scene, cam)
    P = project(scene64(scene), cam, 3)
    u, v, con = P["u"].numpy(), P["v"].numpy(), P["conic"].numpy()
    op, rgb = P["opacity"].numpy(), P["rgb"].numpy()
    rng = np.random.default_rng(0)
    e_sub, e_back = [], []
    for (tx, ty) in [(2, 2), (3, 2)]:
        ids = ostep.tile_list(pidx, tx, ty)
        for py in range(ty * 16, ty * 16 + 16):
            for px in range(tx * 16, tx * 16 + 16):
                a, b = _pixel_errors(ids, u, v, con, op, rgb, px, py, rng.choice([-1.0, 1.0], 3))
                e_sub.append(a)
                e_back.append(b)
    e_sub, e_back = np.concatenate(e_sub), np.concatenate(e_back)
    r_sub, r_back = math.sqrt(np.mean(e_sub ** 2)), math.sqrt(np.mean(e_back ** 2))
    print(f"dL/dalpha float32 RMS error over {e_sub.size} entries: final minus composited "
          f"{r_sub:.2e}, summed from the back {r_back:.2e} (x{r_sub / r_back:.1f})")
    assert e_sub.size > 5000
    assert r_sub < 1e-6 and r_back < 2e-7  # both at float32 rounding level
    assert r_sub > 3 * r_back
