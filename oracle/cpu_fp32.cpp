// CPU baseline: one local-optimisation iteration in float32 on all host
// cores (OpenMP). TEST AND BENCHMARK INFRASTRUCTURE ONLY: the benchmark times
// it as the fair CPU baseline beside the float64 oracle, and a host test checks
// its gradients against the oracle. It shares no code with the CUDA library.
//
// What one call computes (Sec. 3.3 "Local Optimization Kernel" and Supp.
// "Local Optimization Kernel": render only the tiles the active set O^t
// touches, back-propagate into O^t only, Supp. "3DGS Optimization in Changed
// Regions": masked Adam), with the base 3DGS image formation it keeps (Supp.
// "Implementation Details"):
//   per view: project every Gaussian (EWA: Sigma' = J W Sigma W^T J^T + 0.3 I
//   with the tangent clamped to 1.3x the half field of view, conic, radius
//   ceil(3 sqrt(lambda_max)), SH colour max(0, sum + 0.5), sigmoid opacity);
//   the tiles touched by an active Gaussian's rectangle; per such tile the
//   Gaussians whose rectangle holds it in (depth, index) order; per pixel
//   front-to-back compositing (alpha = min(0.99, o exp(power)), skip if
//   power > 0 or alpha < 1/255, stop before an entry when T (1 - alpha) <
//   1e-4); the L1 or L2 loss over the rendered pixels, normalised by
//   3 H W V; per pixel the adjoint with the colour behind each entry summed
//   from the back; the chain rule to the parameters of the active rows.
// The plain algorithm: no pair buckets, no lazy sort, no cached static
// prefix; every list is built and fully sorted every iteration.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <omp.h>

namespace {

struct Cam {  // the layout of the Python side's ctypes structure
    float R[9], t[3], pos[3], fx, fy, cx, cy, znear;
    int32_t W, H;
};

constexpr int kTile = 16;

struct Proj {
    float u, v, z, A, B, C, o, rgb[3];
    int x0, x1, y0, y1;
    bool ok;
};

struct Entry {
    float z;
    int32_t id;
};

// Real spherical harmonics to degree 3 (the base method's sign convention)
// and their gradients with respect to the unit direction.
void sh_eval(float x, float y, float z, int deg, float* Y, float (*dY)[3]) {
    const double PI = 3.14159265358979323846;
    const float c0 = (float)(0.5 / std::sqrt(PI)), c1 = (float)std::sqrt(3.0 / (4.0 * PI));
    const float a0 = (float)(0.5 * std::sqrt(15.0 / PI)), a2 = (float)(0.25 * std::sqrt(5.0 / PI)),
                a4 = (float)(0.25 * std::sqrt(15.0 / PI));
    const float b0 = (float)(-0.25 * std::sqrt(35.0 / (2.0 * PI))),
                b1 = (float)(0.5 * std::sqrt(105.0 / PI)),
                b2 = (float)(-0.25 * std::sqrt(21.0 / (2.0 * PI))),
                b3 = (float)(0.25 * std::sqrt(7.0 / PI)),
                b5 = (float)(0.25 * std::sqrt(105.0 / PI));
    auto set = [&](int k, float val, float gx, float gy, float gz) {
        Y[k] = val;
        dY[k][0] = gx; dY[k][1] = gy; dY[k][2] = gz;
    };
    set(0, c0, 0, 0, 0);
    if (deg < 1) return;
    set(1, -c1 * y, 0, -c1, 0);
    set(2, c1 * z, 0, 0, c1);
    set(3, -c1 * x, -c1, 0, 0);
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    set(4, a0 * x * y, a0 * y, a0 * x, 0);
    set(5, -a0 * y * z, 0, -a0 * z, -a0 * y);
    set(6, a2 * (2 * zz - xx - yy), -2 * a2 * x, -2 * a2 * y, 4 * a2 * z);
    set(7, -a0 * x * z, -a0 * z, 0, -a0 * x);
    set(8, a4 * (xx - yy), 2 * a4 * x, -2 * a4 * y, 0);
    if (deg < 3) return;
    set(9, b0 * y * (3 * xx - yy), b0 * 6 * x * y, b0 * (3 * xx - 3 * yy), 0);
    set(10, b1 * x * y * z, b1 * y * z, b1 * x * z, b1 * x * y);
    set(11, b2 * y * (4 * zz - xx - yy), b2 * (-2 * x * y), b2 * (4 * zz - xx - 3 * yy),
        b2 * 8 * y * z);
    set(12, b3 * z * (2 * zz - 3 * xx - 3 * yy), b3 * (-6 * x * z), b3 * (-6 * y * z),
        b3 * (6 * zz - 3 * xx - 3 * yy));
    set(13, b2 * x * (4 * zz - xx - yy), b2 * (4 * zz - 3 * xx - yy), b2 * (-2 * x * y),
        b2 * 8 * x * z);
    set(14, b5 * z * (xx - yy), b5 * 2 * x * z, b5 * (-2 * y * z), b5 * (xx - yy));
    set(15, b0 * x * (xx - 3 * yy), b0 * (3 * xx - 3 * yy), b0 * (-6 * x * y), 0);
}

// Rotation matrix of a unit quaternion (w, x, y, z), row-major.
void quat_rot(const float* q, float* M) {
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    M[0] = 1 - 2 * (y * y + z * z); M[1] = 2 * (x * y - w * z); M[2] = 2 * (x * z + w * y);
    M[3] = 2 * (x * y + w * z); M[4] = 1 - 2 * (x * x + z * z); M[5] = 2 * (y * z - w * x);
    M[6] = 2 * (x * z - w * y); M[7] = 2 * (y * z + w * x); M[8] = 1 - 2 * (x * x + y * y);
}

struct Geo {  // intermediate values of one projection, kept for the chain rule
    float p[3], qn[4], qlen, s[3], Rq[9], Sig[9], J[6], M[6], cov[3], tx, ty;
    bool clx, cly;
    float d[3], dlen, Y[16], dY[16][3], raw[3];
};

bool project_one(const float* row, int deg, const Cam& c, Proj& P, Geo& g, int Tx, int Ty) {
    P.ok = false;
    const float mx = row[0], my = row[1], mz = row[2];
    for (int k = 0; k < 3; ++k)
        g.p[k] = c.R[3 * k] * mx + c.R[3 * k + 1] * my + c.R[3 * k + 2] * mz + c.t[k];
    const float pz = g.p[2];
    if (!(pz > c.znear)) return false;
    const float* q = row + 8;
    g.qlen = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(g.qlen > 0)) return false;
    for (int k = 0; k < 4; ++k) g.qn[k] = q[k] / g.qlen;
    quat_rot(g.qn, g.Rq);
    for (int k = 0; k < 3; ++k) g.s[k] = std::exp(row[4 + k]);
    float N[9];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) N[3 * i + k] = g.Rq[3 * i + k] * g.s[k];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            g.Sig[3 * i + j] = N[3 * i] * N[3 * j] + N[3 * i + 1] * N[3 * j + 1] +
                               N[3 * i + 2] * N[3 * j + 2];
    const float limx = 1.3f * (0.5f * c.W / c.fx), limy = 1.3f * (0.5f * c.H / c.fy);
    const float xz = g.p[0] / pz, yz = g.p[1] / pz;
    g.clx = xz < -limx || xz > limx;
    g.cly = yz < -limy || yz > limy;
    g.tx = std::min(std::max(xz, -limx), limx) * pz;
    g.ty = std::min(std::max(yz, -limy), limy) * pz;
    g.J[0] = c.fx / pz; g.J[1] = 0; g.J[2] = -c.fx * g.tx / (pz * pz);
    g.J[3] = 0; g.J[4] = c.fy / pz; g.J[5] = -c.fy * g.ty / (pz * pz);
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k)
            g.M[3 * r + k] = g.J[3 * r] * c.R[k] + g.J[3 * r + 1] * c.R[3 + k] +
                             g.J[3 * r + 2] * c.R[6 + k];
    float MS[6];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k)
            MS[3 * r + k] = g.M[3 * r] * g.Sig[k] + g.M[3 * r + 1] * g.Sig[3 + k] +
                            g.M[3 * r + 2] * g.Sig[6 + k];
    const float a = MS[0] * g.M[0] + MS[1] * g.M[1] + MS[2] * g.M[2] + 0.3f;
    const float b = MS[0] * g.M[3] + MS[1] * g.M[4] + MS[2] * g.M[5];
    const float cc = MS[3] * g.M[3] + MS[4] * g.M[4] + MS[5] * g.M[5] + 0.3f;
    g.cov[0] = a; g.cov[1] = b; g.cov[2] = cc;
    const float det = a * cc - b * b;
    if (!(det > 0)) return false;
    const float mid = 0.5f * (a + cc);
    const float lam = mid + std::sqrt(std::max(0.1f, mid * mid - det));
    const float rad = std::ceil(3.0f * std::sqrt(lam));
    P.u = c.fx * xz + c.cx;
    P.v = c.fy * yz + c.cy;
    if (!(P.u == P.u) || !(P.v == P.v)) return false;
    // tile indices clamped in float first (far off-screen centres)
    auto tile_of = [](float x, int hi) {
        return (int)std::min(std::max(std::floor(x / kTile), -1.0f), (float)hi + 1.0f);
    };
    P.x0 = std::max(0, tile_of(P.u - rad, Tx));
    P.x1 = std::min(Tx - 1, tile_of(P.u + rad, Tx));
    P.y0 = std::max(0, tile_of(P.v - rad, Ty));
    P.y1 = std::min(Ty - 1, tile_of(P.v + rad, Ty));
    if (P.x0 > P.x1 || P.y0 > P.y1) return false;
    P.z = pz;
    P.A = cc / det; P.B = -b / det; P.C = a / det;
    P.o = 1.0f / (1.0f + std::exp(-row[3]));
    for (int k = 0; k < 3; ++k) g.d[k] = row[k] - c.pos[k];
    g.dlen = std::sqrt(g.d[0] * g.d[0] + g.d[1] * g.d[1] + g.d[2] * g.d[2]);
    for (int k = 0; k < 3; ++k) g.d[k] /= g.dlen;
    sh_eval(g.d[0], g.d[1], g.d[2], deg, g.Y, g.dY);
    const int K = (deg + 1) * (deg + 1);
    for (int ch = 0; ch < 3; ++ch) {
        float s = 0.5f;
        for (int k = 0; k < K; ++k) s += g.Y[k] * row[12 + 3 * k + ch];
        g.raw[ch] = s;
        P.rgb[ch] = std::max(0.0f, s);
    }
    P.ok = true;
    return true;
}

// Chain rule of one view's 2D gradients (du, dv, dA, dB, dC, do, dr, dg, db)
// to the parameter row's gradient `out` (accumulated).
void chain_rule(const float* row, int deg, const Cam& c, const Geo& g, const float* g2,
                float* out) {
    const float gu = g2[0], gv = g2[1], gA = g2[2], gB = g2[3], gC = g2[4], go = g2[5];
    const float pz = g.p[2];
    float dp[3] = {0, 0, 0};
    // image position
    dp[0] += gu * c.fx / pz;
    dp[1] += gv * c.fy / pz;
    dp[2] += -(gu * c.fx * g.p[0] + gv * c.fy * g.p[1]) / (pz * pz);
    // conic (A, B, C) = inverse of cov [[a, b], [b, c]]: dL/dcov = -Q G Q with
    // G = [[gA, gB/2], [gB/2, gC]] (B is both off-diagonal entries of Q)
    const float a = g.cov[0], b = g.cov[1], cc = g.cov[2];
    const float det = a * cc - b * b;
    const float Q[4] = {cc / det, -b / det, -b / det, a / det};
    const float G[4] = {gA, 0.5f * gB, 0.5f * gB, gC};
    float QG[4], H[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) QG[2 * i + j] = Q[2 * i] * G[j] + Q[2 * i + 1] * G[2 + j];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            H[2 * i + j] = -(QG[2 * i] * Q[j] + QG[2 * i + 1] * Q[2 + j]);
    // cov = M Sig M^T + 0.3 I: dL/dSig = M^T H M, dL/dM = 2 H M Sig
    float dSig[9], HM[6], dM[6];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) HM[3 * r + k] = H[2 * r] * g.M[k] + H[2 * r + 1] * g.M[3 + k];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) dSig[3 * i + j] = g.M[i] * HM[j] + g.M[3 + i] * HM[3 + j];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k)
            dM[3 * r + k] = 2.0f * (HM[3 * r] * g.Sig[k] + HM[3 * r + 1] * g.Sig[3 + k] +
                                    HM[3 * r + 2] * g.Sig[6 + k]);
    // M = J W: dL/dJ = dL/dM W^T
    float dJ[6];
    for (int r = 0; r < 2; ++r)
        for (int i = 0; i < 3; ++i)
            dJ[3 * r + i] = dM[3 * r] * c.R[3 * i] + dM[3 * r + 1] * c.R[3 * i + 1] +
                            dM[3 * r + 2] * c.R[3 * i + 2];
    // J entries: fx/z, -fx tx/z^2, fy/z, -fy ty/z^2 with tx = clamp(x/z) z
    const float z2 = pz * pz, z3 = z2 * pz;
    dp[2] += -c.fx / z2 * dJ[0] - c.fy / z2 * dJ[4];
    dp[2] += 2.0f * c.fx * g.tx / z3 * dJ[2] + 2.0f * c.fy * g.ty / z3 * dJ[5];
    const float dtx = -c.fx / z2 * dJ[2], dty = -c.fy / z2 * dJ[5];
    if (g.clx) dp[2] += dtx * (g.tx / pz); else dp[0] += dtx;
    if (g.cly) dp[2] += dty * (g.ty / pz); else dp[1] += dty;
    // p = W mu + t
    for (int k = 0; k < 3; ++k)
        out[k] += c.R[k] * dp[0] + c.R[3 + k] * dp[1] + c.R[6 + k] * dp[2];
    // Sig = N N^T, N = Rq diag(s)
    float N[9], dN[9];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) N[3 * i + k] = g.Rq[3 * i + k] * g.s[k];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k)
            dN[3 * i + k] = 2.0f * (dSig[3 * i] * N[k] + dSig[3 * i + 1] * N[3 + k] +
                                    dSig[3 * i + 2] * N[6 + k]);
    float dRq[9];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) dRq[3 * i + k] = dN[3 * i + k] * g.s[k];
    for (int k = 0; k < 3; ++k) {
        float ds = 0;
        for (int i = 0; i < 3; ++i) ds += dN[3 * i + k] * g.Rq[3 * i + k];
        out[4 + k] += ds * g.s[k];
    }
    // rotation of the unit quaternion, then its normalisation: per quaternion
    // component, half the derivative of each rotation entry
    const float w = g.qn[0], x = g.qn[1], y = g.qn[2], z = g.qn[3];
    const float half_dR[4][9] = {{0, -z, y, z, 0, -x, -y, x, 0},
                                 {0, y, z, y, -2 * x, -w, z, w, -2 * x},
                                 {-2 * y, x, w, x, 0, z, -w, z, -2 * y},
                                 {-2 * z, -w, x, w, -2 * z, y, x, y, 0}};
    float dq[4];
    for (int k = 0; k < 4; ++k) {
        float acc = 0;
        for (int e = 0; e < 9; ++e) acc += dRq[e] * half_dR[k][e];
        dq[k] = 2 * acc;
    }
    const float dot = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
    for (int k = 0; k < 4; ++k) out[8 + k] += (dq[k] - g.qn[k] * dot) / g.qlen;
    // opacity
    const float o = 1.0f / (1.0f + std::exp(-row[3]));
    out[3] += go * o * (1.0f - o);
    // colour: SH coefficients and the view direction
    const int K = (deg + 1) * (deg + 1);
    float draw[3];
    for (int ch = 0; ch < 3; ++ch) draw[ch] = g.raw[ch] >= 0 ? g2[6 + ch] : 0.0f;
    float dd[3] = {0, 0, 0};
    for (int k = 0; k < K; ++k) {
        float dy = 0;
        for (int ch = 0; ch < 3; ++ch) {
            out[12 + 3 * k + ch] += g.Y[k] * draw[ch];
            dy += row[12 + 3 * k + ch] * draw[ch];
        }
        for (int e = 0; e < 3; ++e) dd[e] += dy * g.dY[k][e];
    }
    const float dd_dot = dd[0] * g.d[0] + dd[1] * g.d[1] + dd[2] * g.d[2];
    for (int e = 0; e < 3; ++e) out[e] += (dd[e] - g.d[e] * dd_dot) / g.dlen;
}

}  // namespace

extern "C" {

// One iteration's forward and backward over V views. rows [n][stride] (the
// library's row layout: mean, opacity logit, log-scale, pad, quaternion, SH
// coefficient-major), active [n] 0/1, cams [V], targets: per view [3][H][W]
// planar, views concatenated. held (optional, per view [H][W], views
// concatenated): pixels whose colour is held constant (no gradient flows
// through them). Writes grads [n][stride] (zero for static rows), image
// (optional, same layout as targets; NaN outside rendered tiles) and the loss
// over rendered pixels. Returns 0, or -1 on bad input.
int cpu_iteration(const float* rows, int32_t n, int32_t stride, int32_t deg,
                  const uint8_t* active, const Cam* cams, int32_t V, const float* targets,
                  int32_t loss_mode, const uint8_t* held, float* grads, float* image,
                  double* loss_out, int32_t threads) {
    if (n < 0 || V <= 0 || deg < 0 || deg > 3 || stride < 12 + 3 * (deg + 1) * (deg + 1) ||
        (loss_mode != 1 && loss_mode != 2))
        return -1;
    if (threads > 0) omp_set_num_threads(threads);
    std::memset(grads, 0, sizeof(float) * (size_t)n * stride);
    std::vector<int32_t> slot(n, -1);
    std::vector<int32_t> act;
    for (int32_t i = 0; i < n; ++i)
        if (active[i]) {
            slot[i] = (int32_t)act.size();
            act.push_back(i);
        }
    const int64_t A = (int64_t)act.size();
    double loss = 0.0;
    std::vector<Proj> P(n);
    std::vector<float> g2(A * 9);
    size_t pix_off = 0;
    for (int j = 0; j < V; ++j) {
        const Cam& c = cams[j];
        const int W = c.W, H = c.H, Tx = (W + kTile - 1) / kTile, Ty = (H + kTile - 1) / kTile;
        const float norm = 1.0f / (3.0f * W * H * V);
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < n; ++i) {
            Geo g;
            project_one(rows + (int64_t)i * stride, deg, c, P[i], g, Tx, Ty);
        }
        // tiles touched by an active Gaussian, and their lists
        std::vector<uint8_t> on(Tx * Ty, 0);
        for (int32_t i : act)
            if (P[i].ok)
                for (int y = P[i].y0; y <= P[i].y1; ++y)
                    for (int x = P[i].x0; x <= P[i].x1; ++x) on[y * Tx + x] = 1;
        std::vector<int64_t> cnt(Tx * Ty + 1, 0);
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < n; ++i) {
            if (!P[i].ok) continue;
            for (int y = P[i].y0; y <= P[i].y1; ++y)
                for (int x = P[i].x0; x <= P[i].x1; ++x)
                    if (on[y * Tx + x]) {
#pragma omp atomic
                        cnt[y * Tx + x + 1]++;
                    }
        }
        for (int t = 0; t < Tx * Ty; ++t) cnt[t + 1] += cnt[t];
        std::vector<Entry> lists(cnt[Tx * Ty]);
        std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < n; ++i) {
            if (!P[i].ok) continue;
            for (int y = P[i].y0; y <= P[i].y1; ++y)
                for (int x = P[i].x0; x <= P[i].x1; ++x)
                    if (on[y * Tx + x]) {
                        int64_t at;
#pragma omp atomic capture
                        at = fill[y * Tx + x]++;
                        lists[at] = Entry{P[i].z, i};
                    }
        }
        std::fill(g2.begin(), g2.end(), 0.0f);
        const float* tgt = targets + 3 * pix_off;
        float* img = image ? image + 3 * pix_off : nullptr;
        if (img)
            for (size_t k = 0; k < (size_t)3 * W * H; ++k) img[k] = NAN;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : loss)
        for (int t = 0; t < Tx * Ty; ++t) {
            if (!on[t]) continue;
            Entry* L = lists.data() + cnt[t];
            const int64_t nl = cnt[t + 1] - cnt[t];
            std::sort(L, L + nl, [](const Entry& a, const Entry& b) {
                return a.z < b.z || (a.z == b.z && a.id < b.id);
            });
            const int tx = t % Tx, ty = t / Tx;
            std::vector<int32_t> used;
            std::vector<float> al, Ts;
            for (int py = ty * kTile; py < std::min(H, ty * kTile + kTile); ++py)
                for (int px = tx * kTile; px < std::min(W, tx * kTile + kTile); ++px) {
                    used.clear(); al.clear(); Ts.clear();
                    float T = 1.0f, C[3] = {0, 0, 0};
                    const float fx = px + 0.5f, fy = py + 0.5f;
                    for (int64_t k = 0; k < nl; ++k) {
                        const Proj& p = P[L[k].id];
                        const float dx = fx - p.u, dy = fy - p.v;
                        const float pw = -0.5f * (p.A * dx * dx + p.C * dy * dy) - p.B * dx * dy;
                        if (pw > 0) continue;
                        const float a = std::min(0.99f, p.o * std::exp(pw));
                        if (a < 1.0f / 255.0f) continue;
                        if (T * (1 - a) < 1e-4f) break;
                        for (int ch = 0; ch < 3; ++ch) C[ch] += p.rgb[ch] * a * T;
                        used.push_back((int32_t)k); al.push_back(a); Ts.push_back(T);
                        T *= 1 - a;
                    }
                    const size_t plane = (size_t)W * H, pi = (size_t)py * W + px;
                    const bool hold = held && held[pix_off + pi];
                    float gch[3];
                    for (int ch = 0; ch < 3; ++ch) {
                        const float dlt = C[ch] - tgt[ch * plane + pi];
                        if (img) img[ch * plane + pi] = C[ch];
                        if (loss_mode == 1) {
                            loss += std::fabs(dlt) * norm;
                            gch[ch] = (float)((dlt > 0) - (dlt < 0)) * norm;
                        } else {
                            loss += dlt * dlt * norm;
                            gch[ch] = 2.0f * dlt * norm;
                        }
                        if (hold) gch[ch] = 0.0f;
                    }
                    // adjoint, back to front: colour behind summed from the back
                    float S[3] = {0, 0, 0};  // background black
                    for (int e = (int)used.size() - 1; e >= 0; --e) {
                        const int id = L[used[e]].id;
                        const Proj& p = P[id];
                        const float a = al[e], Tb = Ts[e];
                        const int s = slot[id];
                        if (s >= 0) {
                            const float dx = fx - p.u, dy = fy - p.v;
                            float dLda = 0;
                            for (int ch = 0; ch < 3; ++ch)
                                dLda += gch[ch] * (Tb * p.rgb[ch] - S[ch] / (1 - a));
                            const bool clamped = p.o * std::exp(
                                -0.5f * (p.A * dx * dx + p.C * dy * dy) - p.B * dx * dy) > 0.99f;
                            float* gs = g2.data() + (int64_t)s * 9;
                            if (!clamped) {
                                const float dpw = dLda * a;
                                const float du = dpw * (p.A * dx + p.B * dy);
                                const float dv = dpw * (p.B * dx + p.C * dy);
#pragma omp atomic
                                gs[0] += du;
#pragma omp atomic
                                gs[1] += dv;
#pragma omp atomic
                                gs[2] += -0.5f * dpw * dx * dx;
#pragma omp atomic
                                gs[3] += -dpw * dx * dy;
#pragma omp atomic
                                gs[4] += -0.5f * dpw * dy * dy;
#pragma omp atomic
                                gs[5] += dLda * a / p.o;
                            }
                            for (int ch = 0; ch < 3; ++ch) {
#pragma omp atomic
                                gs[6 + ch] += a * Tb * gch[ch];
                            }
                        }
                        for (int ch = 0; ch < 3; ++ch) S[ch] += p.rgb[ch] * a * Tb;
                    }
                }
        }
#pragma omp parallel for schedule(static)
        for (int64_t s = 0; s < A; ++s) {
            const int32_t i = act[s];
            const float* gs = g2.data() + s * 9;
            bool any = false;
            for (int k = 0; k < 9; ++k) any |= gs[k] != 0.0f;
            if (!any) continue;
            Geo g;
            Proj p;
            if (!project_one(rows + (int64_t)i * stride, deg, c, p, g, Tx, Ty)) continue;
            chain_rule(rows + (int64_t)i * stride, deg, c, g, gs, grads + (int64_t)i * stride);
        }
        pix_off += (size_t)W * H;
    }
    if (loss_out) *loss_out = loss;
    return 0;
}

// Masked Adam on the active rows (Supp. "3DGS Optimization in Changed
// Regions"), step t (1-based, after this call's increment), bias-corrected.
void cpu_adam(float* rows, float* m, float* v, const float* grads, const uint8_t* active,
              int32_t n, int32_t stride, int32_t t, float lr, float b1, float b2, float eps,
              int32_t threads) {
    if (threads > 0) omp_set_num_threads(threads);
    const float c1 = 1.0f - std::pow(b1, (float)t), c2 = 1.0f - std::pow(b2, (float)t);
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        if (!active[i]) continue;
        for (int k = 0; k < stride; ++k) {
            const int64_t e = (int64_t)i * stride + k;
            const float g = grads[e];
            m[e] = b1 * m[e] + (1 - b1) * g;
            v[e] = b2 * v[e] + (1 - b2) * g * g;
            rows[e] -= lr * (m[e] / c1) / (std::sqrt(v[e] / c2) + eps);
        }
    }
}

}  // extern "C"
