// step.cu -- the batched dynamics step s_{t+1} = f(s_t, u_t, theta) of N
// independent hand-plus-object simulations (Sec. III-A; Algorithm 1, "step
// simulation"), with the contact-sensor readout c_t^(l) of every pad.
//
// One group of G lanes (G = 8, 16 or 32) owns one environment at a time and
// walks the environments grid-stride. Per substep the group
//   1. predicts the velocity under gravity;
//   2. culls hand links against the object's bounding sphere (one ballot);
//   3. tests every (sphere, surviving link) pair, spread over the G lanes,
//      and compacts contacts (gap d < margin) into shared memory by ballot;
//   4. moves each contact into the registers of one lane (CPL per lane) with
//      its lever arm, normal, scalar normal/tangential effective masses and
//      bias folded into a target velocity;
//   5. runs `iters` Jacobi projected-impulse iterations: every contact updates
//      against the same body velocity, then the group sums the impulses and
//      their moments with xor shuffles and recomputes the velocity;
//   6. integrates (symplectic Euler, exact rotation exponential) and adds the
//      contacts' impulses into their sensor pads in a fixed order.
// Nothing here is a dense contraction: the kernel is bound by FP32 issue and
// by the shuffles of step 5.
#include "internal.cuh"

namespace ih {
namespace {

constexpr int kBlock = 128;

template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if constexpr (G == 32) {
        return 0xffffffffu;
    } else {
        const int lane = threadIdx.x & 31;
        return ((1u << G) - 1u) << ((lane / G) * G);
    }
}

template <int G>
__device__ __forceinline__ float group_sum(float v, unsigned mask) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

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
        const float dist = sqrtf(dot(d, d));
        h.n = qrot(q, d * (1.0f / dist));
        h.gap = dist - rs;
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

// sphere against a capsule of axis a + s d, s in [0, L], radius rc
__device__ __forceinline__ Hit hit_capsule(V3 c, float rs, V3 a, V3 d, float L, float rc, Q4 q) {
    const V3 ca = c - a;
    const float t = fminf(fmaxf(dot(ca, d) / L, 0.0f), 1.0f);
    const V3 diff = ca - d * (t * L);
    const float dist = sqrtf(dot(diff, diff));
    Hit h;
    h.t = t;
    h.n = (dist < 1e-9f) ? qrot(q, mk(0, 0, 1)) : diff * (1.0f / dist);
    h.gap = dist - rs - rc;
    return h;
}

__device__ __forceinline__ int pad_of(const DevScene &sc, int l, float t) {
    for (int k = 0; k < sc.n_pads; ++k) {
        if (__ldg(sc.pad_link + k) != l) continue;
        if (l == 0) return k;
        const float s0 = __ldg(sc.pad_s0 + k), s1 = __ldg(sc.pad_s1 + k);
        if (t >= s0 && (t < s1 || s1 >= 1.0f)) return k;
    }
    return -1;
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

template <int G, int CPL>
__global__ void __launch_bounds__(kBlock) step_kernel(const StepArgs a) {
    constexpr int GPB = kBlock / G;   // groups per block
    constexpr int CAP = G * CPL;      // staged contacts per group
    // staging: [0] = lever arm r, gap ; [1] = normal n, (link | pad << 8)
    __shared__ float4 stage[GPB][CAP][2];
    __shared__ float padacc[GPB][IH_MAX_PADS * 3];
    __shared__ unsigned char links[GPB][32];

    const DevScene &sc = a.sc;
    const DevConfig &cfg = a.cfg;
    const int grp = threadIdx.x / G;
    const int g = threadIdx.x % G;
    const unsigned gmask = group_mask<G>();
    const int gshift = (threadIdx.x & 31) / G * G;
    const unsigned gbits = (G == 32) ? 0xffffffffu : ((1u << (G & 31)) - 1u);
    const int ns = cfg.substeps, Lk = sc.n_links, P = sc.n_pads;
    const float h = cfg.h;
    const V3 grav = mk(cfg.gx * h, cfg.gy * h, cfg.gz * h);
    unsigned long long w_pairs = 0, w_contacts = 0, w_citers = 0, w_substeps = 0, w_iters = 0;

    for (int env = blockIdx.x * GPB + grp; env < a.N; env += gridDim.x * GPB) {
        int st = a.status[env];
        const float4 P0 = a.pose[2 * env], P1 = a.pose[2 * env + 1];
        const float4 V0 = a.vel[2 * env], V1 = a.vel[2 * env + 1];
        const float2 th = a.params[env];
        const int shp = a.shape[env];
        const int iters = a.iters[env];
        V3 x = xyz(P0);
        Q4 q = {P1.x, P1.y, P1.z, P1.w};
        V3 v = xyz(V0), w = xyz(V1);
        const float m = th.x, mu = th.y, inv_m = 1.0f / m;
        const int sfirst = __ldg(sc.shape_first + shp), S = __ldg(sc.shape_count + shp);
        const float bound = __ldg(sc.shape_bound + shp);
        S6 Jb;
        Jb.xx = __ldg(sc.shape_jinv + 6 * shp + 0); Jb.yy = __ldg(sc.shape_jinv + 6 * shp + 1);
        Jb.zz = __ldg(sc.shape_jinv + 6 * shp + 2); Jb.xy = __ldg(sc.shape_jinv + 6 * shp + 3);
        Jb.xz = __ldg(sc.shape_jinv + 6 * shp + 4); Jb.yz = __ldg(sc.shape_jinv + 6 * shp + 5);

        for (int fr = 0; fr < a.n_frames; ++fr) {
            for (int k = g; k < 3 * P; k += G) padacc[grp][k] = 0.0f;
            if (st & kDiverged) continue;
            const float4 *tab = a.link_tab + (size_t)(a.frame0 + fr) * (ns + 1) * Lk * kLinkStride;
            for (int s = 0; s < ns; ++s) {
                const float4 *L0 = tab + (size_t)s * Lk * kLinkStride;
                const float4 *L1 = L0 + Lk * kLinkStride;
                const V3 v_pred = v + grav;
                const V3 w_pred = w;
                const M3 R = qmat(q);
                const S6 W = world_inv_inertia(R, Jb, inv_m);

                // -- 2. cull links whose bounding volume the object cannot reach
                unsigned surv = 0;
                for (int base = 0; base < Lk; base += G) {
                    const int l = base + g;
                    bool keep = false;
                    if (l < Lk) {
                        const V3 la = xyz(__ldg(L0 + l * kLinkStride));
                        if (l == 0) {
                            const float4 qq = __ldg(L0 + 2);
                            const V3 cl = qrot_inv({qq.x, qq.y, qq.z, qq.w}, x - la);
                            const V3 k3 = mk(fminf(fmaxf(cl.x, -sc.palm_hx), sc.palm_hx),
                                             fminf(fmaxf(cl.y, -sc.palm_hy), sc.palm_hy),
                                             fminf(fmaxf(cl.z, -sc.palm_hz), sc.palm_hz));
                            const V3 dd = cl - k3;
                            const float reach = bound + cfg.margin;
                            keep = dot(dd, dd) < reach * reach;
                        } else {
                            const V3 ld = xyz(__ldg(L0 + l * kLinkStride + 1));
                            const V3 xa = x - la;
                            const float t = fminf(fmaxf(dot(xa, ld), 0.0f), sc.link_len);
                            const V3 dd = xa - ld * t;
                            const float reach = bound + sc.link_rad + cfg.margin;
                            keep = dot(dd, dd) < reach * reach;
                        }
                    }
                    const unsigned bal = (__ballot_sync(gmask, keep) >> gshift) & gbits;
                    surv |= bal << base;
                }
                const int nsurv = __popc(surv);
                for (int l = g; l < Lk; l += G)
                    if ((surv >> l) & 1u) links[grp][__popc(surv & ((1u << l) - 1u))] = (unsigned char)l;
                __syncwarp(gmask);

                // -- 3. narrowphase over (surviving link, sphere) pairs, compacted by ballot
                int nc = 0;
                const int npairs = nsurv * S;
                int li = 0, j = g;
                while (j >= S && li < nsurv) { j -= S; ++li; }
                for (int p0 = 0; p0 < npairs; p0 += G) {
                    bool hit = false;
                    Hit hh = {0.0f, mk(0, 0, 1), 0.0f};
                    V3 r = mk(0, 0, 0);
                    int l = 0;
                    if (p0 + g < npairs) {
                        l = links[grp][li];
                        const float4 sp = __ldg(sc.spheres + sfirst + j);
                        const V3 cr = mmul(R, xyz(sp));     // centre relative to x
                        const V3 c = x + cr;
                        const float4 A0 = __ldg(L0 + l * kLinkStride);
                        const float4 Aq = __ldg(L0 + l * kLinkStride + 2);
                        const Q4 lq = {Aq.x, Aq.y, Aq.z, Aq.w};
                        if (l == 0) {
                            hh = hit_box(c, sp.w, xyz(A0), lq, sc.palm_hx, sc.palm_hy, sc.palm_hz);
                        } else {
                            const V3 ld = xyz(__ldg(L0 + l * kLinkStride + 1));
                            hh = hit_capsule(c, sp.w, xyz(A0), ld, sc.link_len, sc.link_rad, lq);
                        }
                        hit = hh.gap < cfg.margin;
                        r = cr - hh.n * sp.w;
                    }
                    const unsigned bal = (__ballot_sync(gmask, hit) >> gshift) & gbits;
                    if (hit) {
                        const int idx = nc + __popc(bal & ((1u << g) - 1u));
                        if (idx < CAP) {
                            const int pad = pad_of(sc, l, hh.t);
                            stage[grp][idx][0] = make_float4(r.x, r.y, r.z, hh.gap);
                            stage[grp][idx][1] = make_float4(hh.n.x, hh.n.y, hh.n.z,
                                                             __int_as_float(l | ((pad & 0xff) << 8)));
                        }
                    }
                    nc += __popc(bal);
                    j += G;
                    while (j >= S && li < nsurv) { j -= S; ++li; }
                }
                __syncwarp(gmask);
                w_pairs += npairs;
                w_substeps += 1;
                if (nc > cfg.c_max) {   // more contacts than the per-env capacity
                    st |= IH_ENV_OVERFLOW;
                    nc = 0;
                }
                w_contacts += nc;

                // -- 4. contact setup in registers
                V3 cr_[CPL], cn_[CPL], cc_[CPL], lam_[CPL];
                float ikn_[CPL], ikt_[CPL];
                const float trW = W.xx + W.yy + W.zz;
#pragma unroll
                for (int k = 0; k < CPL; ++k) {
                    const int ci = g + k * G;
                    lam_[k] = mk(0, 0, 0);
                    cr_[k] = mk(0, 0, 0); cn_[k] = mk(0, 0, 1); cc_[k] = mk(0, 0, 0);
                    ikn_[k] = 0.0f; ikt_[k] = 0.0f;
                    if (ci < nc) {
                        const float4 s0 = stage[grp][ci][0], s1 = stage[grp][ci][1];
                        const V3 r = xyz(s0), n = xyz(s1);
                        const int l = __float_as_int(s1.w) & 0xff;
                        // k_n = 1/m + (r x n)^T W (r x n); tr K = 3/m + |r|^2 tr W - r^T W r
                        const V3 rn = cross(r, n);
                        const float kn = inv_m + dot(rn, smul(W, rn));
                        const float trK = 3.0f * inv_m + dot(r, r) * trW - dot(r, smul(W, r));
                        ikn_[k] = 1.0f / kn;
                        ikt_[k] = 2.0f / (trK - kn);
                        const float b = contact_bias(cfg, s0.w);
                        V3 vl = mk(0, 0, 0);
                        if (l != 0) {
                            const float4 A0 = __ldg(L0 + l * kLinkStride), B0 = __ldg(L1 + l * kLinkStride);
                            const float4 Aq = __ldg(L0 + l * kLinkStride + 2), Bq = __ldg(L1 + l * kLinkStride + 2);
                            const Q4 qa = {Aq.x, Aq.y, Aq.z, Aq.w}, qb = {Bq.x, Bq.y, Bq.z, Bq.w};
                            const V3 pl = qrot_inv(qa, (x - xyz(A0)) + r);   // contact in link coords
                            vl = ((xyz(B0) - xyz(A0)) + (qrot(qb, pl) - qrot(qa, pl))) * (1.0f / h);
                        }
                        cr_[k] = r; cn_[k] = n; cc_[k] = vl - n * b;
                    }
                }

                // -- 5. Jacobi projected-impulse iterations
                V3 vv = v_pred, ww = w_pred;
                if (nc > 0) {
                    const float inv_nc = 1.0f / (float)nc;
                    for (int it = 0; it < iters; ++it) {
                        V3 F = mk(0, 0, 0), T = mk(0, 0, 0);
#pragma unroll
                        for (int k = 0; k < CPL; ++k) {
                            if (g + k * G < nc) {
                                const V3 n = cn_[k];
                                const V3 u = vv + cross(ww, cr_[k]) - cc_[k];
                                const float un = dot(u, n);
                                const float l_old = dot(lam_[k], n);
                                const float ln = fmaxf(l_old - un * ikn_[k], 0.0f);
                                V3 lt = (lam_[k] - n * l_old) - (u - n * un) * ikt_[k];
                                const float tn2 = dot(lt, lt);
                                const float lim = mu * ln;
                                if (tn2 > lim * lim) lt = lt * (lim * rsqrtf(tn2));
                                const V3 lp = n * ln + lt;
                                lam_[k] = lam_[k] + (lp - lam_[k]) * inv_nc;
                                F = F + lam_[k];
                                T = T + cross(cr_[k], lam_[k]);
                            }
                        }
                        F.x = group_sum<G>(F.x, gmask); F.y = group_sum<G>(F.y, gmask);
                        F.z = group_sum<G>(F.z, gmask); T.x = group_sum<G>(T.x, gmask);
                        T.y = group_sum<G>(T.y, gmask); T.z = group_sum<G>(T.z, gmask);
                        vv = v_pred + F * inv_m;
                        ww = w_pred + smul(W, T);
                    }
                    w_citers += (unsigned long long)nc * iters;
                    w_iters += iters;
                }
                v = vv;
                w = ww;

                // -- 6. symplectic Euler with the exact rotation exponential
                x = x + v * h;
                {
                    const float wn = sqrtf(dot(w, w));
                    float sn, cs;
                    sincosf(0.5f * wn * h, &sn, &cs);
                    const float kq = (wn > 0.0f) ? sn / wn : 0.5f * h;
                    q = qnorm(qmul({cs, w.x * kq, w.y * kq, w.z * kq}, q));
                }
                // sensor pads: force on the pad by the object is -lambda / h,
                // summed per pad in contact order by the lane that owns the pad
#pragma unroll
                for (int k = 0; k < CPL; ++k) {
                    const int ci = g + k * G;
                    if (ci < nc) {
                        float4 s0 = stage[grp][ci][0];
                        s0.x = lam_[k].x; s0.y = lam_[k].y; s0.z = lam_[k].z;
                        stage[grp][ci][0] = s0;
                    }
                }
                __syncwarp(gmask);
                const float inv_h = 1.0f / h;
                for (int p = g; p < P; p += G) {
                    float fx = 0.0f, fy = 0.0f, fz = 0.0f;
                    for (int ci = 0; ci < nc; ++ci) {
                        const float4 s1 = stage[grp][ci][1];
                        if (((__float_as_int(s1.w) >> 8) & 0xff) != p) continue;
                        const float4 s0 = stage[grp][ci][0];
                        fx -= s0.x * inv_h; fy -= s0.y * inv_h; fz -= s0.z * inv_h;
                    }
                    padacc[grp][3 * p + 0] += fx;
                    padacc[grp][3 * p + 1] += fy;
                    padacc[grp][3 * p + 2] += fz;
                }
                __syncwarp(gmask);
            }
            if (!all_finite(x, q, v, w)) st |= IH_ENV_NONFINITE;
            else if (dot(x, x) > cfg.escape_radius * cfg.escape_radius) st |= IH_ENV_ESCAPED;
        }
        // forces of the last frame, averaged over its substeps
        const float inv_ns = 1.0f / (float)ns;
        float *fo = a.forces + (size_t)env * P * 3;
        __syncwarp(gmask);
        for (int k = g; k < 3 * P; k += G) fo[k] = padacc[grp][k] * inv_ns;
        if (g == 0) {
            a.pose[2 * env] = make_float4(x.x, x.y, x.z, 0.0f);
            a.pose[2 * env + 1] = make_float4(q.w, q.x, q.y, q.z);
            a.vel[2 * env] = make_float4(v.x, v.y, v.z, 0.0f);
            a.vel[2 * env + 1] = make_float4(w.x, w.y, w.z, 0.0f);
            a.status[env] = st;
        }
        __syncwarp(gmask);
    }
    if (g == 0 && a.work) {
        atomicAdd(a.work + 0, w_pairs);
        atomicAdd(a.work + 1, w_contacts);
        atomicAdd(a.work + 2, w_citers);
        atomicAdd(a.work + 3, w_substeps);
        atomicAdd(a.work + 4, w_iters);
    }
}

template <int G, int CPL>
cudaError_t launch_t(const StepArgs &a, int grid, cudaStream_t s) {
    step_kernel<G, CPL><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

int step_variant_max_contacts(const StepVariant &v) { return v.group * v.cpl; }

bool step_variant_supported(const StepVariant &v) {
    if (v.block != kBlock) return false;
    switch (v.group * 100 + v.cpl) {
        case 3202: case 3204: case 3208: case 1604: case 1608: case 808: return true;
        default: return false;
    }
}

cudaError_t launch_step(const StepArgs &a, const StepVariant &v, int grid, cudaStream_t s) {
    switch (v.group * 100 + v.cpl) {
        case 3202: return launch_t<32, 2>(a, grid, s);
        case 3204: return launch_t<32, 4>(a, grid, s);
        case 3208: return launch_t<32, 8>(a, grid, s);
        case 1604: return launch_t<16, 4>(a, grid, s);
        case 1608: return launch_t<16, 8>(a, grid, s);
        case 808: return launch_t<8, 8>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ih
