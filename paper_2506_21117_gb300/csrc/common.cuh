// Device-side helpers shared by the kernels of libclsplat (sm_103a).
//
// Integer-deciding arithmetic (tile rectangles, depth-key bits, change votes)
// is written with the explicitly rounded intrinsics __fadd_rn, __fsub_rn,
// __fmul_rn, __fdiv_rn and __fsqrt_rn, which the compiler never contracts into
// FMAs, so those decisions are one fixed IEEE float32 operation sequence that
// can be reproduced exactly on any IEEE machine. Everything else uses ordinary
// fast float32 arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/clsplat.h"

namespace cls {

constexpr int kTile = CLS_TILE;
constexpr int kTilePixels = kTile * kTile;

inline int64_t hmin64(int64_t a, int64_t b) { return a < b ? a : b; }

// Stream handle of the C ABI is the CUDA runtime's stream handle.
inline cudaStream_t as_stream(cls_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }

// Launch facts that depend on the device (its SM count, the resident blocks of
// a persistent kernel, raised shared-memory limits, which are per device too):
// computed once per device under a lock, so concurrent first calls do not
// race and a device with another SM count or occupancy gets its own value.
// Devices past kMaxDevices compute the value on every call.
constexpr int kMaxDevices = 64;
struct PerDevice {
    std::mutex m;
    int value[kMaxDevices] = {};
};

template <typename F>
inline int per_device(PerDevice& c, F compute) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        dev = 0;
    }
    if (dev < 0 || dev >= kMaxDevices) return compute(dev);
    std::lock_guard<std::mutex> lock(c.m);
    if (c.value[dev] == 0) c.value[dev] = compute(dev);
    return c.value[dev];
}

inline int device_sms(int dev) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Blocks of `kernel` resident on the whole device (persistent grids).
template <typename K>
inline int resident_blocks(int dev, K kernel, int threads, size_t smem) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    return device_sms(dev) * (per_sm > 0 ? per_sm : 1);
}

__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float rsqrt_rn(float a) { return __fsqrt_rn(a); }

// Record a device-side error; CLS_OK is never written so the first error of a
// sequence of launches survives until the caller reads it.
__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
    if (status) atomicCAS(status, CLS_OK, code);
}

// exp(x) in float32 from correctly rounded operations only: Cody & Waite
// reduction x = k ln2 + r with ln2 split into a 12-trailing-zero-bit head and
// a tail, e^r by its Taylor series to degree 7 (|r| <= ln2/2, truncation
// below 2^-27 relative) in Horner form, then the exact scaling by 2^k built
// from exponent bits. The argument is clamped to [-87, 88] so 2^k is normal.
__device__ __forceinline__ float exp_cw(float x) {
    const float kLog2e = (float)1.4426950408889634;
    const float kLn2Hi = 0.693115234375f;  // float(ln 2) with its low 12 bits cleared
    const float kLn2Lo = (float)(0.6931471805599453 - 0.693115234375);
    x = fminf(fmaxf(x, -87.0f), 88.0f);
    const float kf = rintf(rmul(x, kLog2e));
    const float r = rsub(rsub(x, rmul(kf, kLn2Hi)), rmul(kf, kLn2Lo));
    float p = (float)(1.0 / 5040.0);
    p = radd(rmul(p, r), (float)(1.0 / 720.0));
    p = radd(rmul(p, r), (float)(1.0 / 120.0));
    p = radd(rmul(p, r), (float)(1.0 / 24.0));
    p = radd(rmul(p, r), (float)(1.0 / 6.0));
    p = radd(rmul(p, r), 0.5f);
    p = radd(rmul(p, r), 1.0f);
    p = radd(rmul(p, r), 1.0f);
    const float two_k = __int_as_float(((int)kf + 127) << 23);
    return rmul(p, two_k);
}

__device__ __forceinline__ float dot3_rn(float a0, float a1, float a2, float b0, float b1,
                                         float b2) {
    return radd(radd(rmul(a0, b0), rmul(a1, b1)), rmul(a2, b2));
}

// p = R mu + t, each row summed left to right, then t added.
__device__ __forceinline__ void camera_point(const ClsCamera& c, float x, float y, float z,
                                             float& px, float& py, float& pz) {
    px = radd(dot3_rn(c.R[0], c.R[1], c.R[2], x, y, z), c.t[0]);
    py = radd(dot3_rn(c.R[3], c.R[4], c.R[5], x, y, z), c.t[1]);
    pz = radd(dot3_rn(c.R[6], c.R[7], c.R[8], x, y, z), c.t[2]);
}

// Tile rectangle of a projected Gaussian; false if it covers no tile.
__device__ __forceinline__ bool tile_rect(float u, float v, float radius, int tiles_x,
                                          int tiles_y, int& x0, int& x1, int& y0, int& y1) {
    const float ft = (float)kTile;
    const float fx0 = fmaxf(floorf(rdiv(rsub(u, radius), ft)), 0.0f);
    const float fx1 = fminf(floorf(rdiv(radd(u, radius), ft)), (float)(tiles_x - 1));
    const float fy0 = fmaxf(floorf(rdiv(rsub(v, radius), ft)), 0.0f);
    const float fy1 = fminf(floorf(rdiv(radd(v, radius), ft)), (float)(tiles_y - 1));
    if (!(fx0 <= fx1) || !(fy0 <= fy1)) return false;
    x0 = (int)fx0; x1 = (int)fx1; y0 = (int)fy0; y1 = (int)fy1;
    return true;
}

// Projection result of one Gaussian in one view.
struct Proj {
    bool valid;
    float u, v, z, radius;
    float xz, yz;          // p.x / p.z, p.y / p.z
    float px, py, pz;      // camera-space point
    float s[3];            // activated scales
    float qn[4];           // normalised quaternion (w, x, y, z)
    float qnorm;
    float Rq[9];           // rotation matrix of qn
    float Sig[6];          // 3D covariance 00 01 02 11 12 22
    float T[6];            // 2x3 matrix J * R (rows T0, T1)
    float a, b, c;         // 2D covariance (dilated)
    float det;
    bool clamp_x, clamp_y; // tangent clamped inside J
};

// The base 3DGS EWA projection as one fixed sequence of rounded operations.
// `mean` and `log_scale` are the row's float4s [0..3] and [4..7], `quat` [8..11].
__device__ __forceinline__ void project_gaussian(const ClsCamera& cam, float4 mean,
                                                 float4 log_scale, float4 quat, Proj& P) {
    camera_point(cam, mean.x, mean.y, mean.z, P.px, P.py, P.pz);
    P.z = P.pz;
    bool valid = P.pz > cam.znear;
    P.xz = rdiv(P.px, P.pz);
    P.yz = rdiv(P.py, P.pz);
    P.u = radd(rmul(cam.fx, P.xz), cam.cx);
    P.v = radd(rmul(cam.fy, P.yz), cam.cy);

    P.s[0] = exp_cw(log_scale.x);
    P.s[1] = exp_cw(log_scale.y);
    P.s[2] = exp_cw(log_scale.z);
    const float n2 = radd(radd(radd(rmul(quat.x, quat.x), rmul(quat.y, quat.y)),
                               rmul(quat.z, quat.z)), rmul(quat.w, quat.w));
    valid = valid && (n2 > 0.0f);
    const float nrm = rsqrt_rn(n2);
    P.qnorm = nrm;
    const float w = rdiv(quat.x, nrm), x = rdiv(quat.y, nrm), y = rdiv(quat.z, nrm),
                z = rdiv(quat.w, nrm);
    P.qn[0] = w; P.qn[1] = x; P.qn[2] = y; P.qn[3] = z;
    const float xx = rmul(x, x), yy = rmul(y, y), zz = rmul(z, z);
    const float xy = rmul(x, y), xzq = rmul(x, z), yzq = rmul(y, z);
    const float wx = rmul(w, x), wy = rmul(w, y), wz = rmul(w, z);
    float* R = P.Rq;
    R[0] = rsub(1.0f, rmul(2.0f, radd(yy, zz)));
    R[1] = rmul(2.0f, rsub(xy, wz));
    R[2] = rmul(2.0f, radd(xzq, wy));
    R[3] = rmul(2.0f, radd(xy, wz));
    R[4] = rsub(1.0f, rmul(2.0f, radd(xx, zz)));
    R[5] = rmul(2.0f, rsub(yzq, wx));
    R[6] = rmul(2.0f, rsub(xzq, wy));
    R[7] = rmul(2.0f, radd(yzq, wx));
    R[8] = rsub(1.0f, rmul(2.0f, radd(xx, yy)));
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) M[i * 3 + j] = rmul(R[i * 3 + j], P.s[j]);
    }
    P.Sig[0] = dot3_rn(M[0], M[1], M[2], M[0], M[1], M[2]);
    P.Sig[1] = dot3_rn(M[0], M[1], M[2], M[3], M[4], M[5]);
    P.Sig[2] = dot3_rn(M[0], M[1], M[2], M[6], M[7], M[8]);
    P.Sig[3] = dot3_rn(M[3], M[4], M[5], M[3], M[4], M[5]);
    P.Sig[4] = dot3_rn(M[3], M[4], M[5], M[6], M[7], M[8]);
    P.Sig[5] = dot3_rn(M[6], M[7], M[8], M[6], M[7], M[8]);

    const float limx = rmul(1.3f, rdiv(rmul(0.5f, (float)cam.width), cam.fx));
    const float limy = rmul(1.3f, rdiv(rmul(0.5f, (float)cam.height), cam.fy));
    const float txz = fminf(fmaxf(P.xz, -limx), limx);
    const float tyz = fminf(fmaxf(P.yz, -limy), limy);
    P.clamp_x = !(P.xz >= -limx && P.xz <= limx);
    P.clamp_y = !(P.yz >= -limy && P.yz <= limy);
    const float tx = rmul(txz, P.pz);
    const float ty = rmul(tyz, P.pz);
    const float z2 = rmul(P.pz, P.pz);
    const float J00 = rdiv(cam.fx, P.pz);
    const float J02 = -rdiv(rmul(cam.fx, tx), z2);
    const float J11 = rdiv(cam.fy, P.pz);
    const float J12 = -rdiv(rmul(cam.fy, ty), z2);
    const float* W = cam.R;
    float* T = P.T;
    T[0] = radd(rmul(J00, W[0]), rmul(J02, W[6]));
    T[1] = radd(rmul(J00, W[1]), rmul(J02, W[7]));
    T[2] = radd(rmul(J00, W[2]), rmul(J02, W[8]));
    T[3] = radd(rmul(J11, W[3]), rmul(J12, W[6]));
    T[4] = radd(rmul(J11, W[4]), rmul(J12, W[7]));
    T[5] = radd(rmul(J11, W[5]), rmul(J12, W[8]));
    const float* S = P.Sig;  // symmetric: S00 S01 S02 S11 S12 S22
    const float U00 = dot3_rn(T[0], T[1], T[2], S[0], S[1], S[2]);
    const float U01 = dot3_rn(T[0], T[1], T[2], S[1], S[3], S[4]);
    const float U02 = dot3_rn(T[0], T[1], T[2], S[2], S[4], S[5]);
    const float U10 = dot3_rn(T[3], T[4], T[5], S[0], S[1], S[2]);
    const float U11 = dot3_rn(T[3], T[4], T[5], S[1], S[3], S[4]);
    const float U12 = dot3_rn(T[3], T[4], T[5], S[2], S[4], S[5]);
    P.a = radd(dot3_rn(U00, U01, U02, T[0], T[1], T[2]), 0.3f);
    P.b = dot3_rn(U00, U01, U02, T[3], T[4], T[5]);
    P.c = radd(dot3_rn(U10, U11, U12, T[3], T[4], T[5]), 0.3f);
    P.det = rsub(rmul(P.a, P.c), rmul(P.b, P.b));
    valid = valid && (P.det > 0.0f);
    const float mid = rmul(0.5f, radd(P.a, P.c));
    const float disc = rsub(rmul(mid, mid), P.det);
    const float lam = radd(mid, rsqrt_rn(fmaxf(0.1f, disc)));
    P.radius = ceilf(rmul(3.0f, rsqrt_rn(lam)));
    valid = valid && (P.u == P.u) && (P.v == P.v) && (P.radius == P.radius);
    P.valid = valid;
}

// Real SH basis up to degree 3 (base 3DGS sign convention), unit direction.
__device__ __forceinline__ void sh_basis(float x, float y, float z, int degree, float* Y) {
    const float C0 = 0.28209479177387814f;
    const float C1 = 0.4886025119029199f;
    Y[0] = C0;
    if (degree < 1) return;
    Y[1] = -C1 * y; Y[2] = C1 * z; Y[3] = -C1 * x;
    if (degree < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = 1.0925484305920792f * x * y;
    Y[5] = -1.0925484305920792f * y * z;
    Y[6] = 0.31539156525252005f * (2.0f * zz - xx - yy);
    Y[7] = -1.0925484305920792f * x * z;
    Y[8] = 0.5462742152960396f * (xx - yy);
    if (degree < 3) return;
    Y[9] = -0.5900435899266435f * y * (3.0f * xx - yy);
    Y[10] = 2.890611442640554f * x * y * z;
    Y[11] = -0.4570457994644658f * y * (4.0f * zz - xx - yy);
    Y[12] = 0.3731763325901154f * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -0.4570457994644658f * x * (4.0f * zz - xx - yy);
    Y[14] = 1.445305721320277f * z * (xx - yy);
    Y[15] = -0.5900435899266435f * x * (xx - 3.0f * yy);
}

// Alpha of one (pixel, Gaussian) pair, as the forward and backward kernels
// both compute it (so they take identical skip decisions). The conic of a
// staged record is pre-scaled so the exponent comes out in base 2, and the
// opacity o enters the exponent as log2 o (o 2^e = 2^(e + log2 o)):
//   a2 = -A/2 log2(e),  b2 = -B log2(e),  c2 = -C/2 log2(e),  lo = log2 o,
//   power2 = a2 dx^2 + b2 dx dy + c2 dy^2 + lo = power * log2(e) + lo,
//   o G = 2^power2,  alpha = min(0.99, 2^power2),
// so the test power <= 0 reads power2 <= lo. The exponent is formed as
// P + dy (Q + c2 dy) with P = a2 dx^2 + lo and Q = b2 dx computed once per
// entry for the pixels of one column (pair_column).
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float4 stage_conic_a(float4 r0) {  // (u, v, A, B) -> (u, v, a2, b2)
    return make_float4(r0.x, r0.y, -0.5f * kLog2e * r0.z, -kLog2e * r0.w);
}
__device__ __forceinline__ float4 stage_conic_b(float4 r1) {  // (C, o, r, g) -> (c2, lo, r, g)
    return make_float4(-0.5f * kLog2e * r1.x, lg2_approx(r1.y), r1.z, r1.w);
}
__device__ __forceinline__ void pair_column(float dx, float a2, float b2, float lo, float& P,
                                            float& Q) {
    P = __fmaf_rn(a2 * dx, dx, lo);
    Q = b2 * dx;
}
__device__ __forceinline__ float pair_power2(float P, float Q, float dy, float c2) {
    return __fmaf_rn(dy, __fmaf_rn(c2, dy, Q), P);
}
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
// Speculative depth cut (bucketed layout): depth bins emitted beyond the last
// bin a tile needed in the previous iteration.
constexpr int kCutMargin = 4;

// Conservative per-tile cull of a list entry: true only if no pixel centre of
// the tile whose first pixel is (tx0, ty0) can reach alpha >= 1/255, so every
// pixel would skip the entry and dropping it changes nothing. With
// Q(d) = A dx^2 + 2 B dx dy + C dy^2 (the record's conic; power = -Q/2), the
// minimum of Q over the rectangle of the tile's pixel offsets is 0 if the
// centre lies inside, else it lies on an edge, at the stationary point along
// that edge clamped to it. The offsets bound exactly the renderer's own
// dx = (x + 0.5) - u (same rounding, monotone). The bound is lowered by
// 1e-5 S + 1e-5, S >= |A| dx^2 + 2|B dx dy| + |C| dy^2 on the rectangle: both
// this minimum and the renderer's exponent are float32 sums whose rounding is
// near 1e-7 S. An entry is culled if even that lowered minimum leaves
// o exp(-Q/2) below 0.999 / 255.
__device__ __forceinline__ bool tile_culled(float4 r0, float4 r1, float tx0, float ty0) {
    const float u = r0.x, v = r0.y, A = r0.z, B = r0.w, C = r1.x, o = r1.y;
    if (o < kAlphaMin * 0.999f) return true;
    const float X0 = (tx0 + 0.5f) - u, X1 = (tx0 + (float)kTile - 0.5f) - u;
    const float Y0 = (ty0 + 0.5f) - v, Y1 = (ty0 + (float)kTile - 0.5f) - v;
    if (X0 <= 0.f && X1 >= 0.f && Y0 <= 0.f && Y1 >= 0.f) return false;
    const float iA = 1.0f / A, iC = 1.0f / C;
    float q = 3.4e38f;
    {
        const float ya = fminf(fmaxf(-B * X0 * iC, Y0), Y1);
        const float yb = fminf(fmaxf(-B * X1 * iC, Y0), Y1);
        const float xa = fminf(fmaxf(-B * Y0 * iA, X0), X1);
        const float xb = fminf(fmaxf(-B * Y1 * iA, X0), X1);
        q = fminf(q, A * X0 * X0 + 2.0f * B * X0 * ya + C * ya * ya);
        q = fminf(q, A * X1 * X1 + 2.0f * B * X1 * yb + C * yb * yb);
        q = fminf(q, A * xa * xa + 2.0f * B * xa * Y0 + C * Y0 * Y0);
        q = fminf(q, A * xb * xb + 2.0f * B * xb * Y1 + C * Y1 * Y1);
    }
    const float DX = fmaxf(fabsf(X0), fabsf(X1)), DY = fmaxf(fabsf(Y0), fabsf(Y1));
    const float S = (fabsf(A) + fabsf(B)) * DX * DX + (fabsf(B) + fabsf(C)) * DY * DY;
    const float q_lo = q - 1e-5f * S - 1e-5f;
    return q_lo > 2.0f * logf(o * (255.0f / 0.999f));
}

// View index owning a global tile id (views sorted by tile_base).
__device__ __forceinline__ int view_of_tile(const ClsView* views, int n_views, int tile) {
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace cls

// Host-side launch checking shared by the entry points.
#define CLS_CHECK_LAUNCH()                                   \
    do {                                                     \
        if (cudaPeekAtLastError() != cudaSuccess) {          \
            (void)cudaGetLastError();                        \
            return CLS_ERR_CUDA;                             \
        }                                                    \
    } while (0)
