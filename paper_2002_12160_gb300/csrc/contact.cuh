// contact.cuh -- per-contact device arithmetic shared by the forward step
// (step_kernel.cuh, step_pd.cu) and its adjoint (adjoint.cu): narrowphase of a sphere against the
// palm box and a finger capsule, the contact's bias and effective masses, one
// projected Jacobi update, and the 6-value sum over the lanes of a group.
// Both kernels include this header so that the adjoint differentiates exactly
// the arithmetic the step runs.
#pragma once

#include "internal.cuh"

namespace ih {

struct Hit {
    float gap;
    V3 n;     // from the link toward the object
    float t;  // axial fraction along a capsule, 0 on the palm
};

// sphere (centre c, radius rs) against the palm box (pose a, q; half extents)
__device__ __forceinline__ Hit hit_box(V3 c, float rs, V3 a, Q4 q, float hx, float hy, float hz) {
    const V3 cl = qrot_inv(q, c - a);
    const V3 k = mk(fminf(fmaxf(cl.x, -hx), hx), fminf(fmaxf(cl.y, -hy), hy), fminf(fmaxf(cl.z, -hz), hz));
    Hit h;
    h.t = 0.0f;
    const bool inside = (k.x == cl.x) && (k.y == cl.y) && (k.z == cl.z);
    if (!inside) {
        const V3 d = cl - k;
        const float d2 = dot(d, d);
        const float inv = rsqrtf(d2);   // d2 > 0: the centre is outside the box
        h.n = qrot(q, d * inv);
        h.gap = d2 * inv - rs;
    } else {
        // shallowest face, ties to the lowest axis and the + side
        float best = hx - cl.x;
        V3 nl = mk(1, 0, 0);
        if (hx + cl.x < best) { best = hx + cl.x; nl = mk(-1, 0, 0); }
        if (hy - cl.y < best) { best = hy - cl.y; nl = mk(0, 1, 0); }
        if (hy + cl.y < best) { best = hy + cl.y; nl = mk(0, -1, 0); }
        if (hz - cl.z < best) { best = hz - cl.z; nl = mk(0, 0, 1); }
        if (hz + cl.z < best) { best = hz + cl.z; nl = mk(0, 0, -1); }
        h.n = qrot(q, nl);
        h.gap = -best - rs;
    }
    return h;
}

// sphere at ca (relative to the capsule start) against the axis s d, s in [0, L]
__device__ __forceinline__ Hit hit_capsule(V3 ca, float rs, V3 d, float L, float inv_L, float rc, Q4 q) {
    const float t = fminf(fmaxf(dot(ca, d) * inv_L, 0.0f), 1.0f);
    const V3 diff = ca - d * (t * L);
    const float d2 = dot(diff, diff);
    Hit h;
    h.t = t;
    if (d2 < 1e-18f) {   // centre on the axis
        h.n = qrot(q, mk(0, 0, 1));
        h.gap = -rs - rc;
    } else {
        const float inv = rsqrtf(d2);
        h.n = diff * inv;
        h.gap = d2 * inv - rs - rc;
    }
    return h;
}

__device__ __forceinline__ bool link_reaches(const DevScene &sc, const DevConfig &cfg, const float4 *L0,
                                             int l, V3 x, float bound) {
    const V3 la = xyz(__ldg(L0 + l * kLinkStride));
    const V3 xa = x - la;
    if (l == 0) {
        const float4 qq = __ldg(L0 + 2);
        const V3 cl = qrot_inv({qq.x, qq.y, qq.z, qq.w}, xa);
        const V3 k3 = mk(fminf(fmaxf(cl.x, -sc.palm_hx), sc.palm_hx), fminf(fmaxf(cl.y, -sc.palm_hy), sc.palm_hy),
                         fminf(fmaxf(cl.z, -sc.palm_hz), sc.palm_hz));
        const V3 dd = cl - k3;
        const float reach = bound + cfg.margin;
        return dot(dd, dd) < reach * reach;
    }
    const V3 ld = xyz(__ldg(L0 + l * kLinkStride + 1));
    const float t = fminf(fmaxf(dot(xa, ld), 0.0f), sc.link_len);
    const V3 dd = xa - ld * t;
    const float reach = bound + sc.link_rad + cfg.margin;
    return dot(dd, dd) < reach * reach;
}

__device__ __forceinline__ float contact_bias(const DevConfig &cfg, float gap) {
    if (gap > 0.0f) return gap / cfg.h;
    return fmaxf(cfg.beta * fminf(gap + cfg.slop, 0.0f) / cfg.h, -cfg.vmax);
}

__device__ __forceinline__ bool all_finite(V3 x, Q4 q, V3 v, V3 w) {
    return isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(q.w) && isfinite(q.x) &&
           isfinite(q.y) && isfinite(q.z) && isfinite(v.x) && isfinite(v.y) && isfinite(v.z) &&
           isfinite(w.x) && isfinite(w.y) && isfinite(w.z);
}

// Per-contact constants: scalar effective masses along the normal and in the
// tangent plane, and the target velocity c = v_link - b n (bias folded in).
struct CSetup {
    float ikn, ikt;
    V3 cc;
};

__device__ __forceinline__ CSetup setup_contact(V3 r, V3 n, float gap, int l, const S6 &Wi, float trW, float inv_m,
                                                const DevConfig &cfg, const float4 *L0, const float4 *L1, V3 x,
                                                float inv_h) {
    // k_n = 1/m + (r x n)^T W (r x n); tr K = 3/m + |r|^2 tr W - r^T W r
    const V3 rn = cross(r, n);
    const float kn = inv_m + dot(rn, smul(Wi, rn));
    const float trK = 3.0f * inv_m + dot(r, r) * trW - dot(r, smul(Wi, r));
    CSetup c;
    c.ikn = 1.0f / kn;
    c.ikt = 2.0f / (trK - kn);
    const float b = contact_bias(cfg, gap);
    V3 vl = mk(0, 0, 0);
    if (l != 0) {   // link point velocity from the link's rigid displacement over the substep
        const float4 A0 = __ldg(L0 + l * kLinkStride), B0 = __ldg(L1 + l * kLinkStride);
        const float4 Aq = __ldg(L0 + l * kLinkStride + 2), Bq = __ldg(L1 + l * kLinkStride + 2);
        const Q4 qa = {Aq.x, Aq.y, Aq.z, Aq.w}, qb = {Bq.x, Bq.y, Bq.z, Bq.w};
        const V3 pl = qrot_inv(qa, (x - xyz(A0)) + r);   // contact in link coords
        vl = ((xyz(B0) - xyz(A0)) + (qrot(qb, pl) - qrot(qa, pl))) * inv_h;
    }
    c.cc = vl - n * b;
    return c;
}

// One projected Jacobi update of a contact's impulse against the body
// velocity (vv, ww): scalar normal step clamped at zero, scalar tangential
// step clamped radially to the Coulomb disk, relaxed by 1/n_c. The disk clamp
// is a select, not a branch, so that the sliding and the sticking lanes of a
// warp stay in one stretch of code (the same values bit for bit; steps 2-6 %
// faster).
__device__ __forceinline__ V3 update_contact(V3 lam, V3 r, V3 n, V3 cc, float ikn, float ikt, V3 vv, V3 ww,
                                             float mu, float inv_nc) {
    const V3 u = vv + cross(ww, r) - cc;
    const float un = dot(u, n);
    const float l_old = dot(lam, n);
    const float ln = fmaxf(l_old - un * ikn, 0.0f);
    V3 lt = (lam - n * l_old) - (u - n * un) * ikt;
    const float tn2 = dot(lt, lt);
    const float lim = mu * ln;
    const bool slip = tn2 > lim * lim;
    const float sc = lim * rsqrtf(slip ? tn2 : 1.0f);
    lt = lt * (slip ? sc : 1.0f);
    const V3 lp = n * ln + lt;
    return lam + (lp - lam) * inv_nc;
}

// Sum of 6 values over the WIDTH lanes of a group (WIDTH = 16 or 32), every
// lane receiving all 6 sums. Reduce-scatter first: padded to 8 values, each
// of the first three xor levels halves the values a lane keeps (the partner
// sends the half the lane keeps and keeps the other half), the remaining levels
// are plain; the lane at position (k>>2) W/2 + ((k>>1)&1) W/4 + (k&1) W/8
// then holds the full sum of value k, and six shuffles broadcast them.
// 15 shuffles and 9 additions for WIDTH = 32 instead of 30 and 30.
template <int WIDTH>
__device__ __forceinline__ float width_scatter6(const float (&v)[6], unsigned mask, int lane_in_group) {
    const bool b2 = lane_in_group & (WIDTH / 2), b4 = lane_in_group & (WIDTH / 4), b8 = lane_in_group & (WIDTH / 8);
    float a[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float lo = v[i], hi = (i + 4 < 6) ? v[i + 4] : 0.0f;
        const float send = b2 ? lo : hi;
        a[i] = (b2 ? hi : lo) + __shfl_xor_sync(mask, send, WIDTH / 2, WIDTH);
    }
    float b[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = b4 ? a[i] : a[i + 2];
        b[i] = (b4 ? a[i + 2] : a[i]) + __shfl_xor_sync(mask, send, WIDTH / 4, WIDTH);
    }
    float c = (b8 ? b[1] : b[0]) + __shfl_xor_sync(mask, b8 ? b[0] : b[1], WIDTH / 8, WIDTH);
#pragma unroll
    for (int o = WIDTH / 16; o > 0; o >>= 1) c += __shfl_xor_sync(mask, c, o, WIDTH);
    return c;
}
// lane of a group holding value k after width_scatter6
template <int WIDTH>
__device__ __forceinline__ int scatter_lane(int k) {
    return (k >> 2) * (WIDTH / 2) + ((k >> 1) & 1) * (WIDTH / 4) + (k & 1) * (WIDTH / 8);
}

template <int WIDTH>
__device__ __forceinline__ void width_sum6(float (&v)[6], unsigned mask, int lane_in_group) {
    const float c = width_scatter6<WIDTH>(v, mask, lane_in_group);
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = __shfl_sync(mask, c, scatter_lane<WIDTH>(k), WIDTH);
}

}  // namespace ih
