// step_kernel.cuh -- the batched dynamics step s_{t+1} = f(s_t, u_t, theta) of N
// independent hand-plus-object simulations (Sec. III-A; Algorithm 1, "step
// simulation"), with the contact-sensor readout c_t^(l) of every pad.
//
// A group of TPE threads (16, 32, 64 or 128) owns one environment at a time
// and walks the environments grid-stride; groups wider than a warp
// synchronise with named barriers. Per substep the group
//   1. predicts the velocity under gravity and caches the object's spheres,
//      rotated into the world frame, in shared memory;
//   2. culls hand links against the object's bounding sphere (one ballot);
//   3. tests every (surviving link, sphere) pair, TPE pairs per round, and
//      compacts contacts (gap d < margin) into shared memory in pair order by
//      ballot (and, across warps, by per-warp counts);
//   4. moves each contact into the registers of one thread (CPL per thread)
//      with its lever arm, normal, scalar normal/tangential effective masses
//      and the bias folded into a target velocity;
//   5. runs `iters` Jacobi projected-impulse iterations: every contact updates
//      against the same body velocity, then the group sums impulses and
//      moments (xor shuffles, then a double-buffered shared-memory exchange
//      between warps) and recomputes the body velocity;
//   6. integrates (symplectic Euler, exact rotation exponential) and adds the
//      contacts' impulses into their sensor pads in a fixed order, each pad
//      scanning only the contacts of its own link.
// Nothing here is a dense contraction: the kernel is bound by FP32 issue and
// by the latency of the solver's reductions.
#pragma once
#include <cstddef>

#include "contact.cuh"
#include "internal.cuh"

namespace ih {
namespace {

constexpr int kBlock = 128;
// the compiled (group width, register contacts per thread) shapes
#define IH_STEP_VARIANTS(X) X(16, 2) X(16, 4) X(32, 1) X(32, 2) X(32, 3) X(32, 4) X(64, 1) X(64, 2) X(128, 1)
constexpr int kMaxLinks = 32;
constexpr int kPadsPerLink = 4;

template <int TPE>
struct Group {
    static constexpr int GPB = kBlock / TPE;               // groups per block
    static constexpr int W = TPE >= 32 ? TPE / 32 : 1;     // warps per group
    static constexpr int WIDTH = TPE < 32 ? TPE : 32;      // lanes of the group in one warp
    int grp, tid, wid, lane;
    unsigned mask;    // this group's lanes in the warp
    int shift;        // first lane of this group in the warp
    __device__ Group() {
        grp = threadIdx.x / TPE;
        tid = threadIdx.x % TPE;
        lane = threadIdx.x & 31;
        wid = tid / 32;
        if constexpr (TPE < 32) {
            shift = (lane / TPE) * TPE;
            mask = ((1u << TPE) - 1u) << shift;
        } else {
            shift = 0;
            mask = 0xffffffffu;
        }
    }
    __device__ __forceinline__ void sync() const {
        if constexpr (TPE <= 32) {
            __syncwarp(mask);
        } else if constexpr (TPE == kBlock) {
            __syncthreads();
        } else {
            asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(TPE) : "memory");
        }
    }
    // ballot of `p` over the group's lanes in this warp, bit 0 = first lane
    __device__ __forceinline__ unsigned ballot(bool p) const {
        const unsigned b = __ballot_sync(mask, p);
        if constexpr (TPE < 32) return (b >> shift) & ((1u << TPE) - 1u);
        return b;
    }
    __device__ __forceinline__ int lane_in_warp() const { return TPE < 32 ? tid : lane; }
};

// Shared memory of one group. Everything has a fixed size except the contact
// staging, the cache of world-frame sphere and cluster centres and the list of
// surviving (link, cluster) pairs, which follow the group records.

template <int W>
struct alignas(16) GSm {   // 16-byte aligned: red is read as float4
    double term[IH_MAX_PADS];        // FP64 force term of each pad (scoring)
    float padacc[IH_MAX_PADS * 3];
    float red[2][W][8];              // cross-warp partial sums
    int cnt[2][2 * W];               // cross-warp hit counts
    int flag[IH_MAX_PADS];           // contact-state mismatch of each pad (scoring)
    double best_c;                   // best (C, env) of this group so far
    int best_i;
    int next;                        // work-queue slot handed to the group (groups wider than a warp)
    unsigned long long work[6];      // this group's work counters (see sim_work_counters)
    unsigned surv;                   // surviving-link mask
    int n_clp;
    int n_prev;                      // warm start: contacts of the last substep (cache entries)
    unsigned char links[32];         // surviving links in order
    unsigned short lbeg[32], lend[32];   // contact range of each link
};

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }
__host__ __device__ constexpr size_t block_smem_bytes() {
    return align16(kMaxLinks) + align16(kMaxLinks * kPadsPerLink) + 2 * align16(4 * IH_MAX_PADS);
}
template <int W>
__host__ __device__ constexpr size_t gsm_bytes() { return align16(sizeof(GSm<W>)); }
static_assert(sizeof(GSm<1>) % 16 == 0 && sizeof(GSm<2>) % 16 == 0 && sizeof(GSm<4>) % 16 == 0,
              "group records must keep 16-byte alignment");
static_assert(offsetof(GSm<2>, red) % 16 == 0, "red is read as float4");
// dynamic part of a group: the contact staging (4 float4 per contact, the
// first stage_cap contacts; the rest of up to c_max spill to global memory),
// the cache of sphere and cluster centres, for a warm-started solver the cache
// of the last substep's contacts, and the surviving (link, cluster) pairs
__host__ __device__ inline size_t group_dyn_floats4(int s_max, int stage_cap, int c_max, bool warm, int clp_cap) {
    return 4 * (size_t)stage_cap + s_max + 32 + (warm ? (size_t)c_max : 0) + ((size_t)clp_cap * 2 + 15) / 16;
}
// contacts a group stages in shared memory: at least its register-resident
// ones, and 64 (32 for the narrow shapes, eight or more groups to a block,
// whose staging would otherwise cap the blocks an SM holds), at most c_max
__host__ __device__ constexpr int stage_capacity(int rcap, int c_max, int groups_per_block) {
    return c_max < (rcap > (groups_per_block >= 8 ? 32 : 64) ? rcap : (groups_per_block >= 8 ? 32 : 64))
               ? c_max
               : (rcap > (groups_per_block >= 8 ? 32 : 64) ? rcap : (groups_per_block >= 8 ? 32 : 64));
}

template <int TPE>
__device__ __forceinline__ void group_sum6(float (&v)[6], const Group<TPE> &G, float *red, int parity) {
    constexpr int WIDTH = Group<TPE>::WIDTH;
    if constexpr (TPE <= 32) {
        width_sum6<WIDTH>(v, G.mask, G.lane_in_warp() & (WIDTH - 1));
    } else {
        // each warp's sums go straight from the lanes that hold them to shared
        // memory; every thread then adds the W warps' partials in warp order
        constexpr int W = Group<TPE>::W;
        const float c = width_scatter6<32>(v, G.mask, G.lane);
        float *r = red + parity * W * 8;
        const int k = G.lane >> 2;
        if ((G.lane & 3) == 0 && k < 6) r[G.wid * 8 + k] = c;
        G.sync();
        const float4 *r4 = reinterpret_cast<const float4 *>(r);
        float4 lo = r4[0], hi = r4[1];
#pragma unroll
        for (int w = 1; w < W; ++w) {
            const float4 l2 = r4[2 * w], h2 = r4[2 * w + 1];
            lo.x += l2.x; lo.y += l2.y; lo.z += l2.z; lo.w += l2.w;
            hi.x += h2.x; hi.y += h2.y;
        }
        v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w; v[4] = hi.x; v[5] = hi.y;
    }
}

// Resident blocks per SM each shape is compiled for (caps its registers):
// one or two register-resident contacts per thread at 4 blocks (128
// registers: with one contact a cap of 5 blocks spilled and ran 6 % slower on
// large batches), four at 3.
#ifndef IH_STEP_MIN_BLOCKS_CPL2
#define IH_STEP_MIN_BLOCKS_CPL2 4
#endif
template <int TPE, int CPL>
struct MinBlocks {
    static constexpr int value = CPL <= 2 ? IH_STEP_MIN_BLOCKS_CPL2 : (CPL <= 4 ? 3 : 2);
};

template <int TPE, int CPL, bool WARM>
__global__ void __launch_bounds__(kBlock, MinBlocks<TPE, CPL>::value) step_kernel(const StepArgs a, int s_max) {
    using Grp = Group<TPE>;
    constexpr int GPB = Grp::GPB, W = Grp::W, RCAP = TPE * CPL;   // register-resident contacts
    extern __shared__ __align__(16) unsigned char smem[];
    const Grp G;
    const DevScene &sc = a.sc;
    const DevConfig &cfg = a.cfg;
    const int ns = cfg.substeps, Lk = sc.n_links, P = sc.n_pads;
    const float h = cfg.h, inv_h = 1.0f / h, inv_L = 1.0f / sc.link_len;
    const V3 grav = mk(cfg.gx * h, cfg.gy * h, cfg.gz * h);
    // the frame, observation and outputs (from the window descriptor when replayed)
    int frame0 = a.frame0;
    const float *obs = a.obs;
    if (a.win) {
        frame0 = a.win->frame0 + a.win_k;
        obs = a.win->obs ? a.win->obs + (size_t)a.win_k * P * 3 : nullptr;
    }
    const bool window_mode = a.cm_frames != nullptr;   // every frame scored, argmin afterwards
    const bool scored = obs != nullptr;
    const int n_win0 = scored ? *a.n_window : 0;       // frames in the window before this launch
    const int n_win = n_win0 + 1;

    // block-wide tables: the pads of each link (in pad order) and their intervals
    unsigned char *pl_cnt = smem;
    unsigned char *pl_id = smem + align16(kMaxLinks);
    float *p_s0 = reinterpret_cast<float *>(smem + align16(kMaxLinks) + align16(kMaxLinks * kPadsPerLink));
    float *p_s1 = p_s0 + IH_MAX_PADS;
    GSm<W> &S = *reinterpret_cast<GSm<W> *>(smem + block_smem_bytes() + G.grp * gsm_bytes<W>());
    const int cap = cfg.c_max;
    const int SC = a.stage_cap;   // contacts staged in shared memory; the rest spill to global memory
    // contact staging: [0] (r, gap -> 1/k_t), [1] (n, link | pad << 8), [2] (c, 1/k_n), [3] (lambda)
    float4 (*stage)[4] = reinterpret_cast<float4 (*)[4]>(
        reinterpret_cast<float4 *>(smem + block_smem_bytes() + GPB * gsm_bytes<W>()) +
        G.grp * group_dyn_floats4(s_max, SC, cap, WARM, a.clp_cap));
    float4 *sph = &stage[SC][0];
    float4 *clc = sph + s_max;   // cluster centres follow the spheres
    // warm start: final impulse (xyz) and pair id (w, link << 8 | sphere) of the
    // environment's last substep's contacts, in pair order
    float4 *prev = clc + 32;
    // surviving (link index << 8 | cluster) pairs in order
    unsigned short *clp = reinterpret_cast<unsigned short *>(prev + (WARM ? cap : 0));
    // contacts SC .. c_max - 1 of the group's environment: its slot of the spill area
    float4 *spill_g = a.spill ? a.spill + (size_t)(blockIdx.x * GPB + G.grp) * (size_t)(cap - SC) * 4 : nullptr;
    auto cslot = [&](int ci) -> float4 * { return ci < SC ? stage[ci] : spill_g + (size_t)(ci - SC) * 4; };
    constexpr bool warm = WARM;
    if (threadIdx.x < kMaxLinks) {
        int c = 0;
        for (int p = 0; p < P && c < kPadsPerLink; ++p)
            if (__ldg(sc.pad_link + p) == (int)threadIdx.x) pl_id[threadIdx.x * kPadsPerLink + c++] = (unsigned char)p;
        pl_cnt[threadIdx.x] = (unsigned char)c;
    }
    for (int p = threadIdx.x; p < P; p += kBlock) {
        p_s0[p] = __ldg(sc.pad_s0 + p);
        p_s1[p] = __ldg(sc.pad_s1 + p);
    }
    __syncthreads();

    int parity = 0;
    if (G.tid == 0) {
        S.best_c = INFINITY;
        S.best_i = 0x7fffffff;
        for (int k = 0; k < 6; ++k) S.work[k] = 0ull;
    }

    // the next work slot of the group: from the launch's work queue (slots in
    // LPT order, taken one environment at a time by whichever group is free),
    // else grid-stride
    auto fetch = [&](int last) -> int {
        if (!a.queue) return last < 0 ? (int)blockIdx.x * GPB + G.grp : last + (int)gridDim.x * GPB;
        int v = 0;
        if constexpr (TPE <= 32) {
            if (G.tid == 0) v = atomicAdd(a.queue, 1);
            v = __shfl_sync(G.mask, v, G.shift);
        } else {
            if (G.tid == 0) S.next = atomicAdd(a.queue, 1);
            G.sync();   // S.next is written again only after the body's closing barrier
            v = S.next;
        }
        return v;
    };
    for (int slot = fetch(-1); slot < a.N; slot = fetch(slot)) {
        const int env = a.order ? __ldg(a.order + slot) : slot;
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
        const int sfirst = __ldg(sc.shape_first + shp), NS = __ldg(sc.shape_count + shp);
        const float bound = __ldg(sc.shape_bound + shp);
        const int ncl = (NS + kCluster - 1) / kCluster;
        const float inv_ncl = 1.0f / (float)ncl;
        const int cfirst = __ldg(sc.cl_first + shp);
        if (warm) {   // the environment's impulse cache from its previous launch
            const int np = a.cache_n[env];
            if (G.tid == 0) S.n_prev = np;
            for (int k = G.tid; k < np; k += TPE) prev[k] = a.cache[(size_t)env * cap + k];
        }
        double c_sum_env = (window_mode && G.tid == 0) ? a.c_sum[env] : 0.0;
        // cost of the frame just stepped against observation ob (Sec. III-C),
        // FP64 without contraction, pads in order; valid in the group's thread 0
        auto frame_cost = [&](const float *ob, int stt) -> double {
            const float inv_ns_f = 1.0f / (float)ns;
            G.sync();
            const double tau = (double)cfg.tau, wf = (double)cfg.w_force;
            const double tau2 = __dmul_rn(tau, tau);
            for (int p = G.tid; p < P; p += TPE) {
                const double fx = S.padacc[3 * p] * inv_ns_f, fy = S.padacc[3 * p + 1] * inv_ns_f,
                             fz = S.padacc[3 * p + 2] * inv_ns_f;
                const double ox = ob[3 * p], oy = ob[3 * p + 1], oz = ob[3 * p + 2];
                const double dx = __dsub_rn(fx, ox), dy = __dsub_rn(fy, oy), dz = __dsub_rn(fz, oz);
                const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                S.term[p] = __dmul_rn(wf, d2);
                const double ns2 = __dadd_rn(__dadd_rn(__dmul_rn(fx, fx), __dmul_rn(fy, fy)), __dmul_rn(fz, fz));
                const double no2 = __dadd_rn(__dadd_rn(__dmul_rn(ox, ox), __dmul_rn(oy, oy)), __dmul_rn(oz, oz));
                S.flag[p] = (ns2 > tau2) != (no2 > tau2);
            }
            G.sync();
            double c = 0.0;
            if (G.tid == 0) {
                if (stt & kDiverged) {
                    c = INFINITY;
                } else {
                    for (int p = 0; p < P; ++p) {
                        c = __dadd_rn(c, S.term[p]);
                        if (S.flag[p]) c = __dadd_rn(c, (double)cfg.w_contact);
                    }
                }
            }
            G.sync();   // S.term / S.flag are reused by the next frame
            return c;
        };

        for (int fr = 0; fr < a.n_frames; ++fr) {
            for (int k = G.tid; k < 3 * P; k += TPE) S.padacc[k] = 0.0f;
            const float4 *tab = a.link_tab + (size_t)(frame0 + fr) * (ns + 1) * Lk * kLinkStride;
            const bool skip = (st & kDiverged) != 0;   // decided once per frame
            for (int s = 0; s < ns && !skip; ++s) {
                const float4 *L0 = tab + (size_t)s * Lk * kLinkStride;
                const float4 *L1 = L0 + Lk * kLinkStride;
                const V3 v_pred = v + grav;
                const V3 w_pred = w;
                const M3 R = qmat(q);
                S6 Jb;   // inverse unit inertia, re-read (L1) rather than held in registers
                Jb.xx = __ldg(sc.shape_jinv + 6 * shp + 0); Jb.yy = __ldg(sc.shape_jinv + 6 * shp + 1);
                Jb.zz = __ldg(sc.shape_jinv + 6 * shp + 2); Jb.xy = __ldg(sc.shape_jinv + 6 * shp + 3);
                Jb.xz = __ldg(sc.shape_jinv + 6 * shp + 4); Jb.yz = __ldg(sc.shape_jinv + 6 * shp + 5);
                const S6 Wi = world_inv_inertia(R, Jb, inv_m);

                // -- 1. spheres and cluster centres to world (relative to x), cached
                for (int j = G.tid; j < NS; j += TPE) {
                    const float4 sp = __ldg(sc.spheres + sfirst + j);
                    const V3 cr = mmul(R, xyz(sp));
                    sph[j] = make_float4(cr.x, cr.y, cr.z, sp.w);
                }
                for (int k = G.tid; k < ncl; k += TPE) {
                    const float4 cl = __ldg(sc.clusters + cfirst + k);
                    const V3 cr = mmul(R, xyz(cl));
                    clc[k] = make_float4(cr.x, cr.y, cr.z, cl.w);
                }
                // -- 2. cull links whose bounding volume the object cannot reach
                if constexpr (TPE >= 32) {
                    if (G.wid == 0) {
                        const bool keep = G.lane < Lk && link_reaches(sc, cfg, L0, G.lane, x, bound);
                        const unsigned ml = __ballot_sync(0xffffffffu, keep);
                        if (G.lane == 0) S.surv = ml;
                    }
                } else {
                    unsigned ml = 0;
                    for (int base = 0; base < Lk; base += TPE) {
                        const int l = base + G.tid;
                        const bool keep = l < Lk && link_reaches(sc, cfg, L0, l, x, bound);
                        ml |= G.ballot(keep) << base;
                    }
                    if (G.tid == 0) S.surv = ml;
                }
                G.sync();
                const unsigned surv = S.surv;
                const int nsurv = __popc(surv);
                for (int l = G.tid; l < kMaxLinks; l += TPE) {
                    if (l < Lk && ((surv >> l) & 1u)) S.links[__popc(surv & ((1u << l) - 1u))] = (unsigned char)l;
                    S.lbeg[l] = 0;
                    S.lend[l] = 0;
                }
                G.sync();

                // -- 3a. cull (surviving link, cluster) pairs by the clusters' enclosing spheres
                int nclp = 0;
                const int ncpairs = nsurv * ncl;
                for (int p0 = 0; p0 < ncpairs; p0 += TPE) {
                    const int p = p0 + G.tid;
                    bool keep = false;
                    int li = 0, k = 0;
                    if (p < ncpairs) {
                        li = min(max((int)(((float)p + 0.5f) * inv_ncl), 0), nsurv - 1);
                        k = p - li * ncl;
                        const float4 cc = clc[k];
                        keep = link_reaches(sc, cfg, L0, S.links[li], x + xyz(cc), cc.w);
                    }
                    const unsigned bal = G.ballot(keep);
                    int off = nclp, tot;
                    if constexpr (TPE > 32) {
                        int *cb = S.cnt[parity];
                        if (G.lane == 0) cb[G.wid] = __popc(bal);
                        G.sync();
                        tot = 0;
#pragma unroll
                        for (int q2 = 0; q2 < W; ++q2) {
                            const int c = cb[q2];
                            if (q2 < G.wid) off += c;
                            tot += c;
                        }
                        parity ^= 1;
                    } else {
                        tot = __popc(bal);
                    }
                    if (keep) clp[off + __popc(bal & ((1u << G.lane_in_warp()) - 1u))] = (unsigned short)((li << 8) | k);
                    nclp += tot;
                }
                G.sync();

                // -- 3b. narrowphase over the spheres of the surviving pairs, in pair order;
                //        each thread tests two pairs per round (two independent chains)
                int nc = 0;
                const int npairs = nclp * kCluster;
                auto test_pair = [&](int p, Hit &hh, V3 &r, int &l, int &j) -> bool {
                    if (p >= npairs) return false;
                    const int e = clp[p / kCluster];
                    j = (e & 0xff) * kCluster + (p % kCluster);
                    l = S.links[e >> 8];
                    if (j >= NS) return false;
                    const float4 sp = sph[j];
                    const V3 cr = xyz(sp);
                    const float4 A0 = __ldg(L0 + l * kLinkStride);
                    const float4 Aq = __ldg(L0 + l * kLinkStride + 2);
                    const Q4 lq = {Aq.x, Aq.y, Aq.z, Aq.w};
                    if (l == 0) {
                        hh = hit_box(x + cr, sp.w, xyz(A0), lq, sc.palm_hx, sc.palm_hy, sc.palm_hz);
                    } else {
                        const V3 ld = xyz(__ldg(L0 + l * kLinkStride + 1));
                        hh = hit_capsule((x - xyz(A0)) + cr, sp.w, ld, sc.link_len, inv_L, sc.link_rad, lq);
                    }
                    r = cr - hh.n * sp.w;
                    return hh.gap < cfg.margin;
                };
                auto emit = [&](int idx, const Hit &hh, V3 r, int l, int j) {
                    if (idx >= cap) return;
                    int pad = -1;
                    const int npl = pl_cnt[l];
                    for (int k = 0; k < npl; ++k) {
                        const int pp = pl_id[l * kPadsPerLink + k];
                        if (l == 0) { pad = pp; break; }
                        const float s0 = p_s0[pp], s1 = p_s1[pp];
                        if (hh.t >= s0 && (hh.t < s1 || s1 >= 1.0f)) { pad = pp; break; }
                    }
                    float4 *c4 = cslot(idx);
                    c4[0] = make_float4(r.x, r.y, r.z, hh.gap);
                    c4[1] = make_float4(hh.n.x, hh.n.y, hh.n.z, __int_as_float(l | ((pad & 0xff) << 8) | (j << 16)));
                };
                for (int p0 = 0; p0 < npairs; p0 += 2 * TPE) {
                    Hit ha = {0.0f, mk(0, 0, 1), 0.0f}, hb = {0.0f, mk(0, 0, 1), 0.0f};
                    V3 ra = mk(0, 0, 0), rb = mk(0, 0, 0);
                    int la = 0, lb = 0, ja = 0, jb = 0;
                    const bool hit_a = test_pair(p0 + G.tid, ha, ra, la, ja);
                    const bool hit_b = test_pair(p0 + TPE + G.tid, hb, rb, lb, jb);
                    const unsigned bal_a = G.ballot(hit_a), bal_b = G.ballot(hit_b);
                    const unsigned below = (1u << G.lane_in_warp()) - 1u;
                    int off_a = nc, off_b, tot;
                    if constexpr (TPE > 32) {
                        int *cb = &S.cnt[parity][0];   // per warp: hits of the first and second halves
                        if (G.lane == 0) { cb[2 * G.wid] = __popc(bal_a); cb[2 * G.wid + 1] = __popc(bal_b); }
                        G.sync();
                        int tot_a = 0, pre_b = 0, tot_b = 0;
#pragma unroll
                        for (int q2 = 0; q2 < W; ++q2) {
                            const int ca = cb[2 * q2], cbb = cb[2 * q2 + 1];
                            if (q2 < G.wid) { off_a += ca; pre_b += cbb; }
                            tot_a += ca;
                            tot_b += cbb;
                        }
                        off_b = nc + tot_a + pre_b;
                        tot = tot_a + tot_b;
                        parity ^= 1;
                    } else {
                        off_b = nc + __popc(bal_a);
                        tot = __popc(bal_a) + __popc(bal_b);
                    }
                    if (hit_a) emit(off_a + __popc(bal_a & below), ha, ra, la, ja);
                    if (hit_b) emit(off_b + __popc(bal_b & below), hb, rb, lb, jb);
                    nc += tot;
                }
                G.sync();
                if (nc > cfg.c_max) {   // more contacts than the per-env capacity
                    st |= IH_ENV_OVERFLOW;
                    nc = 0;
                }
                if (G.tid == 0) {
                    S.work[0] += (unsigned long long)nclp * kCluster;
                    S.work[1] += nc;
                    S.work[2] += nc > 0 ? (unsigned long long)nc * iters : 0ull;
                    S.work[3] += 1;
                    S.work[4] += nc > 0 ? iters : 0;
                    S.work[5] += ncpairs;
                }

                // -- 4. contact setup: the first TPE*CPL contacts in registers, the rest in
                //       shared memory (and beyond SC in the spill area); the contact
                //       range of each link
                V3 cr_[CPL], cn_[CPL], cc_[CPL], lam_[CPL];
                float ikn_[CPL], ikt_[CPL];
                const float trW = Wi.xx + Wi.yy + Wi.zz;
                // warm start: the impulse of the same pair at the end of the last
                // substep (both lists are in pair order: binary search), else zero
                const int n_prev = warm ? S.n_prev : 0;
                auto warm_lam = [&](float wbits) -> V3 {
                    const int id = (__float_as_int(wbits) & 0xff) << 8 | ((__float_as_int(wbits) >> 16) & 0xff);
                    int lo = 0, hi = n_prev;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (__float_as_int(prev[mid].w) < id) lo = mid + 1; else hi = mid;
                    }
                    if (lo < n_prev && __float_as_int(prev[lo].w) == id) return xyz(prev[lo]);
                    return mk(0, 0, 0);
                };
#pragma unroll
                for (int k = 0; k < CPL; ++k) {
                    const int ci = G.tid + k * TPE;
                    lam_[k] = mk(0, 0, 0);
                    cr_[k] = mk(0, 0, 0); cn_[k] = mk(0, 0, 1); cc_[k] = mk(0, 0, 0);
                    ikn_[k] = 0.0f; ikt_[k] = 0.0f;
                    if (ci < nc) {
                        const float4 s0 = stage[ci][0], s1 = stage[ci][1];
                        const int l = __float_as_int(s1.w) & 0xff;
                        if (ci == 0 || (__float_as_int(stage[ci - 1][1].w) & 0xff) != l) S.lbeg[l] = (unsigned short)ci;
                        if (ci == nc - 1 || (__float_as_int(cslot(ci + 1)[1].w) & 0xff) != l) S.lend[l] = (unsigned short)(ci + 1);
                        const CSetup cs = setup_contact(xyz(s0), xyz(s1), s0.w, l, Wi, trW, inv_m, cfg, L0, L1, x, inv_h);
                        cr_[k] = xyz(s0); cn_[k] = xyz(s1); cc_[k] = cs.cc; ikn_[k] = cs.ikn; ikt_[k] = cs.ikt;
                        if (warm) lam_[k] = warm_lam(s1.w);
                    }
                }
                for (int ci = RCAP + G.tid; ci < nc; ci += TPE) {
                    float4 *c4 = cslot(ci);
                    const float4 s0 = c4[0], s1 = c4[1];
                    const int l = __float_as_int(s1.w) & 0xff;
                    if ((__float_as_int(cslot(ci - 1)[1].w) & 0xff) != l) S.lbeg[l] = (unsigned short)ci;
                    if (ci == nc - 1 || (__float_as_int(cslot(ci + 1)[1].w) & 0xff) != l) S.lend[l] = (unsigned short)(ci + 1);
                    const CSetup cs = setup_contact(xyz(s0), xyz(s1), s0.w, l, Wi, trW, inv_m, cfg, L0, L1, x, inv_h);
                    c4[0].w = cs.ikt;
                    c4[2] = make_float4(cs.cc.x, cs.cc.y, cs.cc.z, cs.ikn);
                    const V3 l0 = warm ? warm_lam(s1.w) : mk(0, 0, 0);
                    c4[3] = make_float4(l0.x, l0.y, l0.z, 0.0f);
                }

                // -- 5. Jacobi projected-impulse iterations
                V3 vv = v_pred, ww = w_pred;
                if (nc > 0) {
                    const float inv_nc = 1.0f / (float)nc;
                    const int slot_off = TPE > 32 ? 32 * G.wid : 0;   // this warp's first contact of a slot
                    if (warm) {   // the cached impulses act from the first iteration on
                        float acc[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
                        for (int k = 0; k < CPL; ++k) {
                            if (k * TPE + slot_off < nc) {
                                const V3 tq = cross(cr_[k], lam_[k]);
                                acc[0] += lam_[k].x; acc[1] += lam_[k].y; acc[2] += lam_[k].z;
                                acc[3] += tq.x; acc[4] += tq.y; acc[5] += tq.z;
                            }
                        }
                        for (int ci = RCAP + G.tid; ci < nc; ci += TPE) {
                            const float4 *c4 = cslot(ci);
                            const V3 lam = xyz(c4[3]), tq = cross(xyz(c4[0]), lam);
                            acc[0] += lam.x; acc[1] += lam.y; acc[2] += lam.z;
                            acc[3] += tq.x; acc[4] += tq.y; acc[5] += tq.z;
                        }
                        group_sum6<TPE>(acc, G, &S.red[0][0][0], parity);
                        parity ^= 1;
                        vv = v_pred + mk(acc[0], acc[1], acc[2]) * inv_m;
                        ww = w_pred + smul(Wi, mk(acc[3], acc[4], acc[5]));
                    }
                    for (int it = 0; it < iters; ++it) {
                        float acc[6] = {0, 0, 0, 0, 0, 0};
                        // a register slot is skipped only when it is empty in every
                        // lane of the warp (a warp-uniform branch: in a wider group the
                        // warps holding only empty slots skip it and free issue slots);
                        // otherwise all lanes update it without a branch so the slots'
                        // chains interleave:
                        // an empty slot (r = c = 0, n = z, 1/k = 0, lambda = 0) keeps
                        // lambda = 0 and adds zeros
#pragma unroll
                        for (int k = 0; k < CPL; ++k) {
                            if (k * TPE + slot_off < nc) {
                                lam_[k] = update_contact(lam_[k], cr_[k], cn_[k], cc_[k], ikn_[k], ikt_[k], vv, ww, mu, inv_nc);
                                const V3 tq = cross(cr_[k], lam_[k]);
                                acc[0] += lam_[k].x; acc[1] += lam_[k].y; acc[2] += lam_[k].z;
                                acc[3] += tq.x; acc[4] += tq.y; acc[5] += tq.z;
                            }
                        }
                        // staged contacts: shared memory, then the spill area (this
                        // lane's sequence RCAP + tid, + TPE, ... continued past SC)
                        const int ncs = min(nc, SC);
                        for (int ci = RCAP + G.tid; ci < ncs; ci += TPE) {
                            const float4 s0 = stage[ci][0], s1 = stage[ci][1], s2 = stage[ci][2], s3 = stage[ci][3];
                            const V3 lam = update_contact(xyz(s3), xyz(s0), xyz(s1), xyz(s2), s2.w, s0.w, vv, ww, mu, inv_nc);
                            stage[ci][3] = make_float4(lam.x, lam.y, lam.z, 0.0f);
                            const V3 tq = cross(xyz(s0), lam);
                            acc[0] += lam.x; acc[1] += lam.y; acc[2] += lam.z;
                            acc[3] += tq.x; acc[4] += tq.y; acc[5] += tq.z;
                        }
                        if (nc > SC) {
                            int ci = RCAP + G.tid;
                            if (ci < SC) ci += ((SC - ci + TPE - 1) / TPE) * TPE;
                            for (; ci < nc; ci += TPE) {
                                float4 *c4 = spill_g + (size_t)(ci - SC) * 4;
                                const float4 s0 = c4[0], s1 = c4[1], s2 = c4[2], s3 = c4[3];
                                const V3 lam = update_contact(xyz(s3), xyz(s0), xyz(s1), xyz(s2), s2.w, s0.w, vv, ww, mu, inv_nc);
                                c4[3] = make_float4(lam.x, lam.y, lam.z, 0.0f);
                                const V3 tq = cross(xyz(s0), lam);
                                acc[0] += lam.x; acc[1] += lam.y; acc[2] += lam.z;
                                acc[3] += tq.x; acc[4] += tq.y; acc[5] += tq.z;
                            }
                        }
                        group_sum6<TPE>(acc, G, &S.red[0][0][0], parity);
                        parity ^= 1;
                        vv = v_pred + mk(acc[0], acc[1], acc[2]) * inv_m;
                        ww = w_pred + smul(Wi, mk(acc[3], acc[4], acc[5]));
                    }
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
                // summed over the contacts of the pad's link in contact order
#pragma unroll
                for (int k = 0; k < CPL; ++k) {
                    const int ci = G.tid + k * TPE;
                    if (ci < nc) cslot(ci)[3] = make_float4(lam_[k].x, lam_[k].y, lam_[k].z, 0.0f);
                }
                G.sync();
                for (int p = G.tid; p < P; p += TPE) {
                    const int l = __ldg(sc.pad_link + p);
                    float fx = 0.0f, fy = 0.0f, fz = 0.0f;
                    const int e = S.lend[l];
                    for (int ci = S.lbeg[l]; ci < e; ++ci) {
                        const float4 *c4 = cslot(ci);
                        if (((__float_as_int(c4[1].w) >> 8) & 0xff) != p) continue;
                        const float4 s3 = c4[3];
                        fx -= s3.x * inv_h; fy -= s3.y * inv_h; fz -= s3.z * inv_h;
                    }
                    S.padacc[3 * p + 0] += fx;
                    S.padacc[3 * p + 1] += fy;
                    S.padacc[3 * p + 2] += fz;
                }
                if (warm) {   // this substep's contacts and final impulses, for the next one
                    for (int ci = G.tid; ci < nc; ci += TPE) {
                        const float4 *c4 = cslot(ci);
                        const int wb = __float_as_int(c4[1].w);
                        const float4 l3 = c4[3];
                        prev[ci] = make_float4(l3.x, l3.y, l3.z, __int_as_float((wb & 0xff) << 8 | ((wb >> 16) & 0xff)));
                    }
                    if (G.tid == 0) S.n_prev = nc;
                }
                G.sync();
            }
            if (!skip) {
                if (!all_finite(x, q, v, w)) st |= IH_ENV_NONFINITE;
                else if (dot(x, x) > cfg.escape_radius * cfg.escape_radius) st |= IH_ENV_ESCAPED;
            }
            if (window_mode) {   // this frame's cost, window sum and mean, and pose
                const double c = frame_cost(obs + (size_t)fr * P * 3, st);
                if (G.tid == 0) {
                    c_sum_env = __dadd_rn(c_sum_env, c);
                    const double cm = __ddiv_rn(c_sum_env, (double)(n_win0 + fr + 1));
                    a.cm_frames[(size_t)fr * a.N + env] = cm;
                    float4 *pf = a.pose_frames + 2 * ((size_t)fr * a.N + env);
                    pf[0] = make_float4(x.x, x.y, x.z, 0.0f);
                    pf[1] = make_float4(q.w, q.x, q.y, q.z);
                    if (fr == a.n_frames - 1) {
                        a.c_sum[env] = c_sum_env;
                        a.c_mean[env] = cm;
                        if (a.cost_mean) a.cost_mean[env] = cm;
                    }
                }
            }
        }
        // frame cost against the observation (Sec. III-C), FP64, in pad order,
        // on exactly the forces written out below
        if (scored && !window_mode) {
            const double c = frame_cost(obs, st);
            if (G.tid == 0) {
                const double sum = __dadd_rn(a.c_sum[env], c);
                a.c_sum[env] = sum;
                double cm = __ddiv_rn(sum, (double)n_win);
                a.c_mean[env] = cm;
                if (a.cost_mean) a.cost_mean[env] = cm;
                if (isnan(cm)) cm = INFINITY;
                if (cm < S.best_c || (cm == S.best_c && env < S.best_i)) { S.best_c = cm; S.best_i = env; }
            }
        }
        // forces of the last frame, averaged over its substeps
        const float inv_ns = 1.0f / (float)ns;
        float *fo = a.forces + (size_t)env * P * 3;
        G.sync();
        for (int k = G.tid; k < 3 * P; k += TPE) fo[k] = S.padacc[k] * inv_ns;
        if (G.tid == 0) {
            a.pose[2 * env] = make_float4(x.x, x.y, x.z, 0.0f);
            a.pose[2 * env + 1] = make_float4(q.w, q.x, q.y, q.z);
            a.vel[2 * env] = make_float4(v.x, v.y, v.z, 0.0f);
            a.vel[2 * env + 1] = make_float4(w.x, w.y, w.z, 0.0f);
            a.status[env] = st;
        }
        if (warm) {   // the cache for the next launch
            const int np = S.n_prev;
            if (G.tid == 0) a.cache_n[env] = np;
            for (int k = G.tid; k < np; k += TPE) a.cache[(size_t)env * cap + k] = prev[k];
        }
        G.sync();
    }
    if (G.tid == 0 && a.work)
        for (int k = 0; k < 6; ++k)
            if (S.work[k]) atomicAdd(a.work + k, S.work[k]);
    if (a.queue) {   // the last block to finish empties the queue for the next launch
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();   // this block's queue draws, before its finish ticket
            if (atomicAdd(a.queue + 1, 1) == (int)gridDim.x - 1) {
                atomicExch(a.queue, 0);
                atomicExch(a.queue + 1, 0);
            }
        }
    }
    if (!scored || window_mode) return;
    // argmin (C_i, i) over the grid: per-block candidate, then the last block
    __shared__ bool last;
    __shared__ int best_env;
    __threadfence();   // this thread's pose/status/cost writes, before the ticket
    __syncthreads();
    if (threadIdx.x == 0) {
        double bc = INFINITY;
        int bi = 0x7fffffff;
        for (int g2 = 0; g2 < GPB; ++g2) {
            const GSm<W> &S2 = *reinterpret_cast<const GSm<W> *>(smem + block_smem_bytes() + g2 * gsm_bytes<W>());
            const double c = S2.best_c;
            const int i = S2.best_i;
            if (c < bc || (c == bc && i < bi)) { bc = c; bi = i; }
        }
        a.part_c[blockIdx.x] = bc;
        a.part_i[blockIdx.x] = bi;
        __threadfence();
        last = atomicAdd(a.done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < 32) {
        double bc = INFINITY;
        int bi = 0x7fffffff;
        for (int b = threadIdx.x; b < gridDim.x; b += 32) {
            const double c = __ldcg(a.part_c + b);
            const int i = __ldcg(a.part_i + b);
            if (c < bc || (c == bc && i < bi)) { bc = c; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double oc = __shfl_xor_sync(0xffffffffu, bc, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (oc < bc || (oc == bc && oi < bi)) { bc = oc; bi = oi; }
        }
        if (threadIdx.x == 0) {
            const int best = (bi == 0x7fffffff) ? 0 : bi;
            int *argmin_out = a.argmin_out;
            if (a.win) argmin_out = a.win->argmin ? a.win->argmin + a.win_k : nullptr;
            *a.argmin_state = best;
            if (argmin_out) *argmin_out = best;
            *a.n_window = n_win;
            *a.done = 0u;
            best_env = best;
        }
    }
    __syncthreads();
    float *est_out = a.est_pose_out;
    if (a.win) est_out = a.win->est ? a.win->est + 8 * a.win_k : nullptr;
    if (est_out && threadIdx.x < 8) {
        const float4 p = __ldcg(a.pose + 2 * best_env + (threadIdx.x >> 2));
        const float v[4] = {p.x, p.y, p.z, p.w};
        est_out[threadIdx.x] = v[threadIdx.x & 3];
    }
}

template <int TPE, int CPL, bool WARM>
size_t bytes_t(int s_max, int c_max, int clp_cap) {
    constexpr int GPB = Group<TPE>::GPB;
    const int sc = stage_capacity(TPE * CPL, c_max, GPB);
    return block_smem_bytes() + GPB * gsm_bytes<Group<TPE>::W>() +
           GPB * group_dyn_floats4(s_max, sc, c_max, WARM, clp_cap) * sizeof(float4);
}

// Shared-memory opt-in, and the blocks of this shape that fit on one SM
template <int TPE, int CPL, bool WARM>
cudaError_t prepare_t(int s_max, int c_max, int clp_cap, int *blocks_per_sm) {
    const size_t bytes = bytes_t<TPE, CPL, WARM>(s_max, c_max, clp_cap);
    cudaError_t e = cudaSuccess;
    if (bytes > 48 * 1024)
        e = cudaFuncSetAttribute(step_kernel<TPE, CPL, WARM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && blocks_per_sm)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, step_kernel<TPE, CPL, WARM>, kBlock, bytes);
    return e;
}

template <int TPE, int CPL, bool WARM>
cudaError_t launch_t(const StepArgs &a, int grid, int s_max, cudaStream_t s) {
    step_kernel<TPE, CPL, WARM><<<grid, kBlock, bytes_t<TPE, CPL, WARM>(s_max, a.cfg.c_max, a.clp_cap), s>>>(a, s_max);
    return cudaGetLastError();
}

// The dispatch over the compiled shapes, for the cold (WARM = false) or the
// warm-started (WARM = true) solver; each is instantiated in its own
// translation unit so the two build in parallel.
template <bool WARM>
size_t smem_bytes_w(const StepVariant &v, int s_max, int c_max, int clp_cap) {
#define IH_BYTES(T, C) if (v.group == T && v.cpl == C) return bytes_t<T, C, WARM>(s_max, c_max, clp_cap);
    IH_STEP_VARIANTS(IH_BYTES)
#undef IH_BYTES
    return 0;
}

template <bool WARM>
cudaError_t prepare_w(const StepVariant &v, int s_max, int c_max, int clp_cap, int *blocks_per_sm) {
#define IH_PREP(T, C) if (v.group == T && v.cpl == C) return prepare_t<T, C, WARM>(s_max, c_max, clp_cap, blocks_per_sm);
    IH_STEP_VARIANTS(IH_PREP)
#undef IH_PREP
    return cudaErrorInvalidValue;
}

template <bool WARM>
cudaError_t launch_w(const StepArgs &a, const StepVariant &v, int grid, int s_max, cudaStream_t s) {
#define IH_LAUNCH(T, C) if (v.group == T && v.cpl == C) return launch_t<T, C, WARM>(a, grid, s_max, s);
    IH_STEP_VARIANTS(IH_LAUNCH)
#undef IH_LAUNCH
    return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace ih
