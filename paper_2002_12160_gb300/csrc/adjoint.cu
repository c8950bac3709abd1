// adjoint.cu -- reverse-mode derivative of the tracking cost with respect to
// each environment's initial pose, mass and friction coefficient.
//
// The cost of one environment over the frames [frame0, frame0 + H) is
//     L = sum_f sum_l w_force |c_f^(l) - o_f^(l)|^2  (+ contact-state terms)
// -- the tracking cost of Sec. III-C on the simulated pad forces c_f of the
// frame step s_{t+1} = f(s_t, u_t, theta) of Sec. III-A. The contact-state
// terms are piecewise constant and carry no derivative. The gradient is taken
// by hand-written reverse mode through every operation of the step: sphere
// positions, narrowphase gaps, normals and lever arms, effective masses, bias
// and link velocities, the fixed number of projected Jacobi iterations, and
// the integrator (the same arithmetic as step_kernel.cuh, through contact.cuh).
//
// The projections of the Jacobi update are not differentiable on the cone's
// boundary. The reverse sweep therefore uses smooth stand-ins for their
// derivatives only; the forward values stay exact:
//   * normal clamp max(0, z): the derivative sigmoid(beta z) of a softplus;
//   * radial clamp of the tangential impulse z onto the disk of radius L:
//     the derivative of z smin(|z|, L) / |z| with
//     smin(a, b) = (a + b - sqrt((a - b)^2 + (w b)^2)) / 2.
// Contact membership (gap < margin), the capsule's end clamps, the palm's face
// or clamp pattern and the bias regimes are held fixed.
//
// Work layout: a group of GW warps (32 GW threads) per environment. The
// group enumerates the contacts together, in the step's order; thread
// k % (32 GW) then owns contact k for the setup, the Jacobi iterations and
// their reverse -- its first PL contacts in registers, the further ones in the
// environment's scratch memory -- and the group sums impulses and derivatives
// by warp shuffles and a shared-memory exchange between its warps. The state
// at every K-th frame is kept (checkpoints). The reverse sweep walks the
// segments between checkpoints backwards: it recomputes the segment's
// substep start states and pad forces from its checkpoint while recording the
// tape (the impulses after every Jacobi iteration and the per-iteration
// impulse sums) of every substep of the segment, then runs the substeps'
// reverse sweeps in reverse order. When the whole segment's tape does not fit
// the handle's budget, each substep is run once more just before its reverse
// sweep to record its tape alone; the results are the same bit for bit. (The
// last segment's tape is recorded by the first pass itself.) Checkpoints,
// segment states and the tape live in a slice of a scratch buffer owned by
// the handle, one slice per environment.
#include "contact.cuh"
#include "internal.cuh"

namespace ih {
namespace {

constexpr int kAW = 4;   // warps per CTA
constexpr int kABlock = 32 * kAW;
constexpr unsigned kFull = 0xffffffffu;

// The GW warps of one environment: group thread gt, lane, warp within the
// group, group within the block; sync() is the group's barrier.
template <int GW>
struct AGroup {
    static constexpr int T = 32 * GW;
    int gt, lane, wg, gid;
    __device__ AGroup() {
        gt = threadIdx.x % T;
        lane = threadIdx.x & 31;
        wg = gt >> 5;
        gid = threadIdx.x / T;
    }
    __device__ __forceinline__ void sync() const {
        if constexpr (GW == 1) {
            __syncwarp();
        } else if constexpr (T == kABlock) {
            __syncthreads();
        } else {
            asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(T) : "memory");
        }
    }
};

struct Body {
    V3 x;
    Q4 q;
    V3 v, w;
};
struct Adj {   // derivatives of the cost w.r.t. a Body's components
    V3 x;
    Q4 q;
    V3 v, w;
};

__device__ __forceinline__ void store_body(float4 *p, const Body &b) {
    p[0] = make_float4(b.x.x, b.x.y, b.x.z, 0.0f);
    p[1] = make_float4(b.q.w, b.q.x, b.q.y, b.q.z);
    p[2] = make_float4(b.v.x, b.v.y, b.v.z, 0.0f);
    p[3] = make_float4(b.w.x, b.w.y, b.w.z, 0.0f);
}
__device__ __forceinline__ Body load_body(const float4 *p) {
    const float4 a = p[0], b = p[1], c = p[2], d = p[3];
    return Body{xyz(a), Q4{b.x, b.y, b.z, b.w}, xyz(c), xyz(d)};
}
__device__ __forceinline__ Q4 qconj(Q4 q) { return {q.w, -q.x, -q.y, -q.z}; }

template <int GW>
struct alignas(16) GroupSm {
    // contacts whose record (besides the slot's global one, which the tape
    // keeps) the forward substep also holds here: the register slots' and more
    static constexpr int kRC = GW == 1 ? 64 : 128;
    float4 crec[kRC][2];           // (r, gap), (n, link | pad << 8 as int bits)
    float4 clam[kRC];              // the pass's final impulses of the register slots (pad sums)
    float4 sph[IH_MAX_SPHERES];    // the substep's sphere centres (world rotation, relative to x), radius
    float4 clc[IH_MAX_SPHERES / kCluster];   // cluster centres (likewise), enclosing radius
    double term[IH_MAX_PADS];      // a frame's FP64 force term of each pad
    float padacc[IH_MAX_PADS * 3];
    float fbar[IH_MAX_PADS * 3];   // dL/dF_p / (h ns): minus the derivative w.r.t. a final impulse
    float red[2][GW][8];           // partial sums of the group's warps (double-buffered)
    int cnt[2][GW];                // hits of each warp in a compaction round (double-buffered)
    int flag[IH_MAX_PADS];         // a frame's contact-state mismatch of each pad
    unsigned short lbeg[32], lend[32];
    unsigned short clp[32 * (IH_MAX_SPHERES / kCluster)];   // surviving (link index << 8 | cluster) pairs
    unsigned char links[32];       // surviving links in order
    unsigned surv;
};

// Block-wide pad tables: the pads of each link (in pad order) and their intervals.
constexpr int kAPadsPerLink = 4;
struct PadTab {
    unsigned char cnt[32];
    unsigned char id[32 * kAPadsPerLink];
    float s0[IH_MAX_PADS], s1[IH_MAX_PADS];
};

// Positions of the group's hits in a round of order-preserving compaction:
// `hit` of this thread; returns its slot (base + hits of the threads before
// it in the group) and adds the round's hits to `base`.
template <int GW>
__device__ __forceinline__ int gcompact(bool hit, int &base, const AGroup<GW> &G, GroupSm<GW> &S, int &parity) {
    const unsigned bal = __ballot_sync(kFull, hit);
    int off = base + __popc(bal & ((1u << G.lane) - 1u));
    if constexpr (GW == 1) {
        base += __popc(bal);
    } else {
        int *c = S.cnt[parity];
        if (G.lane == 0) c[G.wg] = __popc(bal);
        G.sync();
        int tot = 0;
#pragma unroll
        for (int w = 0; w < GW; ++w) {
            const int k = c[w];
            if (w < G.wg) off += k;
            tot += k;
        }
        base += tot;
        parity ^= 1;
    }
    return off;
}

// Sum of 6 values over the group's threads, every thread receiving the sums:
// within each warp by shuffles, then the warps' partials in warp order.
template <int GW>
__device__ __forceinline__ void gsum6(float (&v)[6], const AGroup<GW> &G, GroupSm<GW> &S, int &parity) {
    if constexpr (GW == 1) {
        width_sum6<32>(v, kFull, G.lane);
    } else {
        const float c = width_scatter6<32>(v, kFull, G.lane);
        float *r = &S.red[parity][0][0];
        const int k = G.lane >> 2;
        if ((G.lane & 3) == 0 && k < 6) r[G.wg * 8 + k] = c;
        G.sync();
#pragma unroll
        for (int q = 0; q < 6; ++q) v[q] = r[q];
#pragma unroll
        for (int w = 1; w < GW; ++w)
#pragma unroll
            for (int q = 0; q < 6; ++q) v[q] += r[w * 8 + q];
        parity ^= 1;
    }
}

// Per-slot scratch layout in floats (every part starts on a float4 boundary):
// checkpoints, a segment's substep start states, every frame's pad forces, the
// impulses of a pass (final ones for the pad sums; the running ones of the
// contacts past the register slots), the reverse state of the contacts past
// the register slots, the contact count of every taped substep, the contact
// records and counts of the nrec substeps of the segments that are
// recomputed (their recomputation replays them), then nblk tape blocks of
// (contact records, impulse after each iteration, iteration sums): one block
// per substep of a segment when the whole segment is taped, else a single
// block re-filled substep by substep.
struct SlotLayout {
    size_t ck, sg, sf, lamf, adj, ncs, recs, nrc, tape, blk_rec, blk_lamh, blk_sh, blk_stride, total;
};
__host__ __device__ inline size_t round4(size_t x) { return (x + 3) & ~size_t(3); }
__host__ __device__ inline SlotLayout slot_layout(int H, int K, int ns, int P, int cap, int iters_max, int nblk,
                                                  int nrec) {
    SlotLayout L;
    size_t o = 0;
    const size_t nck = (size_t)((H + K - 1) / K);
    L.ck = o;   o += round4(nck * 16);                        // checkpoint states
    L.sg = o;   o += round4((size_t)K * ns * 16);             // substep start states of a segment
    L.sf = o;   o += round4((size_t)H * P * 3);               // pad forces of every frame
    L.lamf = o; o += round4((size_t)cap * 4);                 // impulses of a pass
    L.adj = o;  o += round4((size_t)cap * 16);                // reverse state of the contacts in memory
    L.ncs = o;  o += round4((size_t)K * ns);                  // contacts of each taped substep (int)
    L.recs = o; o += (size_t)nrec * cap * 16;                 // records of the recomputed segments' substeps
    L.nrc = o;  o += round4((size_t)nrec);                    // their contact counts (int)
    L.blk_rec = 0;
    L.blk_lamh = round4((size_t)cap * 16);                                   // contact records
    L.blk_sh = L.blk_lamh + round4((size_t)iters_max * cap * 4);             // impulse after each iteration
    L.blk_stride = L.blk_sh + round4((size_t)(iters_max > 0 ? iters_max : 1) * 8);   // sums after each iteration
    L.tape = o; o += (size_t)nblk * L.blk_stride;
    L.total = o;
    return L;
}

struct SlotPtr {
    float4 *ck, *sg, *rec, *lamh, *lamf;
    float4 *recs;   // records of substep q of the recomputed segments at recs + q * cap * 4
    int *nrc;       // their contact counts
    float4 *adjs;   // per contact past the register slots: (lb, 1/k_n bar), (nb, 1/k_t bar), (rb, -), (cb, -)
    float *sf, *sh;
    int *ncs;
    float *tape;
    size_t blk_lamh, blk_sh, blk_stride;
    // the same slot with its tape pointers on block b
    __device__ SlotPtr blk(int b) const {
        SlotPtr q = *this;
        float *t = tape + (size_t)b * blk_stride;
        q.rec = reinterpret_cast<float4 *>(t);
        q.lamh = reinterpret_cast<float4 *>(t + blk_lamh);
        q.sh = t + blk_sh;
        return q;
    }
};

// Per-environment constants.
struct Env {
    int sfirst, NS, iters, cfirst;
    float mu, inv_m, bound;
    S6 Jb;
};

// contact record: [0] (r, gap) [1] (n, 1/k_n) [2] (c, 1/k_t) [3] (t, link | pad << 8, sphere, -)
__device__ __forceinline__ int rec_link(float4 r3) { return __float_as_int(r3.y) & 0xff; }
__device__ __forceinline__ int rec_pad(float4 r3) { return (__float_as_int(r3.y) >> 8) & 0xff; }

// One substep of one environment (the arithmetic of step_kernel.cuh, contacts in the
// same order: link, then sphere), its contact records written at sp.rec.
// With TAPE the impulses after every iteration and the iteration sums are
// recorded in the slot's current tape block; with PADS the pad forces of the
// substep are added to S.padacc; with replay_nc >= 0 the substep's records
// at sp.rec are those of an earlier run from the same state (replay_nc
// contacts, setup included), which replaces the enumeration and the setup.
// Returns the contact count (0 on overflow). Not inlined, with the flags as
// arguments: every pass (cost, recomputation, tape) then runs the same
// compiled arithmetic, so a recorded tape is bit for bit the forward's.
template <int GW, int PL>
__device__ __noinline__ int fwd_substep(const AdjArgs &a, const Env &E_, Body &b, const float4 *L0,
                                        const float4 *L1, const SlotPtr &sp_, GroupSm<GW> &S, const PadTab &PT,
                                        const AGroup<GW> &G_, int &parity_, int &st_, int tape_flag,
                                        int pads_flag, int replay_nc) {
    // the flags are run-time values (the callers combine them with a.zero):
    // one compiled body serves the cost pass, the recomputation and the tape,
    // so a recorded tape is bit for bit the forward's
    const bool TAPE = tape_flag != 0, PADS = pads_flag != 0;
    static_assert(AGroup<GW>::T * PL <= GroupSm<GW>::kRC, "the register slots' records are in shared memory");
    // by-value copies of what the loops read: through the references every
    // store to the tape or to shared memory could alias them and force reloads
    const Env E = E_;
    const SlotPtr sp = sp_;
    const AGroup<GW> G = G_;
    int parity = parity_, st = st_;
    constexpr int T = AGroup<GW>::T;
    const DevScene sc = a.sc;   // by value, as E below
    const DevConfig cfg = a.cfg;
    const int Lk = sc.n_links, P = sc.n_pads, cap = cfg.c_max;
    const float h = cfg.h, inv_h = 1.0f / h, inv_L = 1.0f / sc.link_len;
    const V3 grav = mk(cfg.gx * h, cfg.gy * h, cfg.gz * h);
    const V3 v_pred = b.v + grav;
    const V3 w_pred = b.w;
    const M3 R = qmat(b.q);
    const S6 Wi = world_inv_inertia(R, E.Jb, E.inv_m);
    const int lane = G.lane;

    const int gt = G.gt;
    int nc = 0;
    const bool replay = replay_nc >= 0;
    if (replay) {
        // the records this substep's first run left, setup included: no
        // enumeration (the run is deterministic, so they are its own)
        nc = replay_nc;
        for (int ci = gt; ci < nc && ci < GroupSm<GW>::kRC; ci += T) {
            const float4 *rc = sp.rec + 4 * ci;
            const float4 r0 = rc[0], r1 = rc[1], r3 = rc[3];
            S.crec[ci][0] = r0;
            S.crec[ci][1] = make_float4(r1.x, r1.y, r1.z, r3.y);
        }
        for (int l = gt; l < 32; l += T) {
            S.lbeg[l] = 0;
            S.lend[l] = 0;
        }
        G.sync();
    } else {
        // contact enumeration by the whole group, in the step's order (link,
        // then sphere): sphere and cluster centres to world, the link cull, the
        // (link, cluster) cull by the clusters' enclosing spheres, then the
        // spheres of the surviving pairs, one test per thread per round,
        // compacted in order
        const int ncl = (E.NS + kCluster - 1) / kCluster;
        for (int j = gt; j < E.NS; j += T) {
            const float4 s4 = __ldg(sc.spheres + E.sfirst + j);
            const V3 cr = mmul(R, xyz(s4));
            S.sph[j] = make_float4(cr.x, cr.y, cr.z, s4.w);
        }
        for (int k = gt; k < ncl; k += T) {
            const float4 cl = __ldg(sc.clusters + E.cfirst + k);
            const V3 cr = mmul(R, xyz(cl));
            S.clc[k] = make_float4(cr.x, cr.y, cr.z, cl.w);
        }
        if (G.wg == 0) {
            const bool keep = lane < Lk && link_reaches(sc, cfg, L0, lane, b.x, E.bound);
            const unsigned surv = __ballot_sync(kFull, keep);
            if (keep) S.links[__popc(surv & ((1u << lane) - 1u))] = (unsigned char)lane;
            if (lane == 0) S.surv = surv;
        }
        for (int l = gt; l < 32; l += T) {
            S.lbeg[l] = 0;
            S.lend[l] = 0;
        }
        G.sync();
        const int ncp = __popc(S.surv) * ncl;
        int nclp = 0;
        for (int p0 = 0; p0 < ncp; p0 += T) {
            const int p = p0 + gt;
            bool keep = false;
            int li = 0, k = 0;
            if (p < ncp) {
                li = p / ncl;
                k = p - li * ncl;
                const float4 cc = S.clc[k];
                keep = link_reaches(sc, cfg, L0, S.links[li], b.x + xyz(cc), cc.w);
            }
            const int off = gcompact<GW>(keep, nclp, G, S, parity);
            if (keep) S.clp[off] = (unsigned short)((li << 8) | k);
        }
        G.sync();
        const int npairs = nclp * kCluster;
        for (int p0 = 0; p0 < npairs; p0 += T) {
            const int p = p0 + gt;
            bool hit = false;
            Hit hh = {0.0f, mk(0, 0, 1), 0.0f};
            V3 r = mk(0, 0, 0);
            int l = 0, j = 0;
            if (p < npairs) {
                const int e = S.clp[p / kCluster];
                j = (e & 0xff) * kCluster + (p % kCluster);
                l = S.links[e >> 8];
                if (j < E.NS) {   // (j >= NS: padding of the shape's last cluster)
                    const float4 s4 = S.sph[j];
                    const V3 cr = xyz(s4);
                    const float4 A0 = __ldg(L0 + l * kLinkStride);
                    const float4 Aq = __ldg(L0 + l * kLinkStride + 2);
                    const Q4 lq = {Aq.x, Aq.y, Aq.z, Aq.w};
                    if (l == 0) {
                        hh = hit_box(b.x + cr, s4.w, xyz(A0), lq, sc.palm_hx, sc.palm_hy, sc.palm_hz);
                    } else {
                        const V3 ld = xyz(__ldg(L0 + l * kLinkStride + 1));
                        hh = hit_capsule((b.x - xyz(A0)) + cr, s4.w, ld, sc.link_len, inv_L, sc.link_rad, lq);
                    }
                    r = cr - hh.n * s4.w;
                    hit = hh.gap < cfg.margin;
                }
            }
            const int idx = gcompact<GW>(hit, nc, G, S, parity);
            if (hit && idx < cap) {
                int pad = -1;   // the first pad of the link whose interval holds t
                const int npl = PT.cnt[l];
                for (int k = 0; k < npl; ++k) {
                    const int pp = PT.id[l * kAPadsPerLink + k];
                    if (l == 0) { pad = pp; break; }
                    const float s0 = PT.s0[pp], s1 = PT.s1[pp];
                    if (hh.t >= s0 && (hh.t < s1 || s1 >= 1.0f)) { pad = pp; break; }
                }
                float4 *rc = sp.rec + 4 * idx;
                const float4 a0 = make_float4(r.x, r.y, r.z, hh.gap);
                const float lp = __int_as_float(l | ((pad & 0xff) << 8));
                rc[0] = a0;
                rc[1] = make_float4(hh.n.x, hh.n.y, hh.n.z, 0.0f);
                rc[3] = make_float4(hh.t, lp, __int_as_float(j), 0.0f);
                if (idx < GroupSm<GW>::kRC) {
                    S.crec[idx][0] = a0;
                    S.crec[idx][1] = make_float4(hh.n.x, hh.n.y, hh.n.z, lp);
                }
            }
        }
        G.sync();   // the records are written
        if (nc > cap) {   // more contacts than the per-env capacity: as the step, no contacts
            st |= IH_ENV_OVERFLOW;
            nc = 0;
        }
    }
    // each link's contact range (the contacts are in link order)
    constexpr int RC = GroupSm<GW>::kRC;
    auto link_of = [&](int c) -> int {
        return c < RC ? (__float_as_int(S.crec[c][1].w) & 0xff) : rec_link(sp.rec[4 * c + 3]);
    };
    for (int ci = gt; ci < nc; ci += T) {
        const int l = link_of(ci);
        if (ci == 0 || link_of(ci - 1) != l) S.lbeg[l] = (unsigned short)ci;
        if (ci == nc - 1 || link_of(ci + 1) != l) S.lend[l] = (unsigned short)(ci + 1);
    }
    G.sync();

    // contact setup, by the thread that owns the contact from here on; the
    // constants stay in its registers for the iterations
    const float trW = Wi.xx + Wi.yy + Wi.zz;
    V3 lam_[PL], cr_[PL], cn_[PL], cc_[PL];
    float ikn_[PL], ikt_[PL];
#pragma unroll
    for (int k = 0; k < PL; ++k) {
        lam_[k] = mk(0, 0, 0);
        cr_[k] = mk(0, 0, 0); cn_[k] = mk(0, 0, 1); cc_[k] = mk(0, 0, 0);
        ikn_[k] = ikt_[k] = 0.0f;
        const int ci = G.gt + T * k;
        if (ci < nc && replay) {   // the setup's results are in the records
            const float4 *rc = sp.rec + 4 * ci;
            const float4 r0 = rc[0], r1 = rc[1], r2 = rc[2];
            cr_[k] = xyz(r0); cn_[k] = xyz(r1); cc_[k] = xyz(r2); ikn_[k] = r1.w; ikt_[k] = r2.w;
        } else if (ci < nc) {   // (a register slot's record is in shared memory: T PL <= kRC)
            float4 *rc = sp.rec + 4 * ci;
            const float4 r0 = S.crec[ci][0], r1 = S.crec[ci][1];
            const CSetup cs = setup_contact(xyz(r0), xyz(r1), r0.w, __float_as_int(r1.w) & 0xff, Wi, trW, E.inv_m, cfg,
                                            L0, L1, b.x, inv_h);
            rc[1] = make_float4(r1.x, r1.y, r1.z, cs.ikn);
            rc[2] = make_float4(cs.cc.x, cs.cc.y, cs.cc.z, cs.ikt);
            cr_[k] = xyz(r0); cn_[k] = xyz(r1); cc_[k] = cs.cc; ikn_[k] = cs.ikn; ikt_[k] = cs.ikt;
        }
    }
    // contacts past the register slots (thread gt's slots PL, PL + 1, ... in
    // the same order): constants in their records, impulse in sp.lamf
    for (int ci = G.gt + T * PL; ci < nc; ci += T) {
        if (!replay) {
            float4 *rc = sp.rec + 4 * ci;
            const float4 r0 = rc[0], r1 = rc[1], r3 = rc[3];
            const CSetup cs = setup_contact(xyz(r0), xyz(r1), r0.w, rec_link(r3), Wi, trW, E.inv_m, cfg, L0, L1, b.x,
                                            inv_h);
            rc[1] = make_float4(r1.x, r1.y, r1.z, cs.ikn);
            rc[2] = make_float4(cs.cc.x, cs.cc.y, cs.cc.z, cs.ikt);
        }
        sp.lamf[ci] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }

    // Jacobi projected-impulse iterations
    V3 vv = v_pred, ww = w_pred;
    if (nc > 0) {
        const float inv_nc = 1.0f / (float)nc;
        for (int it = 0; it < E.iters; ++it) {
            float acc[6] = {0, 0, 0, 0, 0, 0};
            // every register slot without a branch, so that the slots' chains
            // interleave: an empty slot (r = c = 0, n = z, 1/k = 0) keeps a zero
            // impulse and adds zeros
#pragma unroll
            for (int k = 0; k < PL; ++k) {
                const int ci = G.gt + T * k;
                lam_[k] = update_contact(lam_[k], cr_[k], cn_[k], cc_[k], ikn_[k], ikt_[k], vv, ww, E.mu, inv_nc);
                const V3 tq = cross(cr_[k], lam_[k]);
                acc[0] += lam_[k].x; acc[1] += lam_[k].y; acc[2] += lam_[k].z;
                acc[3] += tq.x; acc[4] += tq.y; acc[5] += tq.z;
                if (TAPE && ci < nc) sp.lamh[(size_t)it * cap + ci] = make_float4(lam_[k].x, lam_[k].y, lam_[k].z, 0.0f);
            }
            for (int ci = G.gt + T * PL; ci < nc; ci += T) {
                const float4 *rc = sp.rec + 4 * ci;
                const float4 r0 = rc[0], r1 = rc[1], r2 = rc[2];
                const V3 lam = update_contact(xyz(sp.lamf[ci]), xyz(r0), xyz(r1), xyz(r2), r1.w, r2.w, vv, ww, E.mu,
                                              inv_nc);
                sp.lamf[ci] = make_float4(lam.x, lam.y, lam.z, 0.0f);
                const V3 tq = cross(xyz(r0), lam);
                acc[0] += lam.x; acc[1] += lam.y; acc[2] += lam.z;
                acc[3] += tq.x; acc[4] += tq.y; acc[5] += tq.z;
                if (TAPE) sp.lamh[(size_t)it * cap + ci] = make_float4(lam.x, lam.y, lam.z, 0.0f);
            }
            gsum6<GW>(acc, G, S, parity);
            if (TAPE && G.gt == 0)
                for (int q = 0; q < 6; ++q) sp.sh[8 * it + q] = acc[q];
            vv = v_pred + mk(acc[0], acc[1], acc[2]) * E.inv_m;
            ww = w_pred + smul(Wi, mk(acc[3], acc[4], acc[5]));
        }
    }
    b.v = vv;
    b.w = ww;
    b.x = b.x + b.v * h;
    {
        const float wn = sqrtf(dot(b.w, b.w));
        float sn, cs;
        sincosf(0.5f * wn * h, &sn, &cs);
        const float kq = (wn > 0.0f) ? sn / wn : 0.5f * h;
        b.q = qnorm(qmul({cs, b.w.x * kq, b.w.y * kq, b.w.z * kq}, b.q));
    }
    if (PADS) {
        // pad forces -lambda / h, each pad summing the contacts of its link in
        // order (the contacts past the register slots have theirs in sp.lamf)
#pragma unroll
        for (int k = 0; k < PL; ++k) {
            const int ci = G.gt + T * k;
            if (ci < nc) S.clam[ci] = make_float4(lam_[k].x, lam_[k].y, lam_[k].z, 0.0f);
        }
        G.sync();
        if (G.gt < P && nc > 0) {
            const int l = __ldg(sc.pad_link + lane);
            float fx = 0.0f, fy = 0.0f, fz = 0.0f;
            const int e = S.lend[l];
            for (int ci = S.lbeg[l]; ci < e; ++ci) {
                const int pd = ci < RC ? ((__float_as_int(S.crec[ci][1].w) >> 8) & 0xff) : rec_pad(sp.rec[4 * ci + 3]);
                if (pd != lane) continue;
                const float4 lf = ci < T * PL ? S.clam[ci] : sp.lamf[ci];
                fx -= lf.x * inv_h; fy -= lf.y * inv_h; fz -= lf.z * inv_h;
            }
            S.padacc[3 * lane + 0] += fx;
            S.padacc[3 * lane + 1] += fy;
            S.padacc[3 * lane + 2] += fz;
        }
    }
    G.sync();
    parity_ = parity;
    st_ = st;
    return nc;
}

// d bias / d gap (contact_bias: gap / h when separated, else the clamped
// Baumgarte term)
__device__ __forceinline__ float bias_slope(const DevConfig &cfg, float gap) {
    if (gap > 0.0f) return 1.0f / cfg.h;
    const float z = gap + cfg.slop;
    if (!(z < 0.0f)) return 0.0f;
    return (cfg.beta * z / cfg.h > -cfg.vmax) ? cfg.beta / cfg.h : 0.0f;
}

// The reverse sweep's smoothing functions use the hardware's approximate
// exponential, reciprocal and reciprocal square root (a few ulp each): they
// sit at the head of every reverse iteration's dependent chain, and their
// error is far inside the gradient's tolerance against the FP64 adjoint.
__device__ __forceinline__ float sigmoid(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }

// Reverse of the smoothed radial clamp out = z smin(|z|, L) / |z| for the
// incoming derivative g: returns dL/dz and dL/dL. At z = 0 exactly the
// derivative of the exact clamp inside the disk (identity) is used. With
// Q = sqrt((a - L)^2 + (w L)^2), smin(a, L) = (a + L - Q) / 2 is evaluated as
// L (4a - w^2 L) / (2 (a + L + Q)), the same value without the cancellation
// of a + L - Q when the clamp does not bind (a << L).
__device__ __forceinline__ void disk_bwd(V3 z, float L, V3 g, float w, V3 &zb, float &Lb) {
    const float a2z = dot(z, z);
    const bool at0 = !(a2z > 0.0f);
    const float a2 = at0 ? 1.0f : a2z;   // (without a branch: the values at z = 0 are selected below)
    const float ia = rsqrtf(a2);
    const float a = a2 * ia;
    const float dl = a - L;
    const float wL = w * L;
    const float Q2 = fmaf(dl, dl, wL * wL);
    const float iQ = rsqrtf(Q2);
    const float Q = Q2 * iQ;
    const float phi = __fdividef(L * fmaf(-w, wL, 4.0f * a), 2.0f * (a + L + Q));
    const float pa = 0.5f * (1.0f - dl * iQ);
    const float pb = 0.5f * (1.0f + (dl - w * wL) * iQ);
    const V3 zh = z * ia;
    const float s = dot(zh, g);
    const float ra = phi * ia;
    zb = at0 ? ((L > 0.0f) ? g : mk(0, 0, 0)) : g * ra + zh * (s * (pa - ra));
    Lb = at0 ? 0.0f : s * pb;
}

// Reverse of the narrowphase (hit_box / hit_capsule) for the sphere centred
// at x + cr: the derivative w.r.t. the centre given those w.r.t. gap and n.
__device__ __forceinline__ V3 hit_bwd(const DevScene &sc, int l, V3 x, V3 cr, const float4 *L0, float gb, V3 nb) {
    const float4 A0 = __ldg(L0 + l * kLinkStride);
    const float4 Aq = __ldg(L0 + l * kLinkStride + 2);
    const Q4 q = {Aq.x, Aq.y, Aq.z, Aq.w};
    if (l == 0) {
        const float hx = sc.palm_hx, hy = sc.palm_hy, hz = sc.palm_hz;
        const V3 cl = qrot_inv(q, (x + cr) - xyz(A0));
        const V3 k = mk(fminf(fmaxf(cl.x, -hx), hx), fminf(fmaxf(cl.y, -hy), hy), fminf(fmaxf(cl.z, -hz), hz));
        V3 clb = mk(0, 0, 0);
        if (!((k.x == cl.x) && (k.y == cl.y) && (k.z == cl.z))) {
            const V3 d = cl - k;
            const float inv = rsqrtf(dot(d, d));
            const V3 nl = d * inv;
            const V3 nlb = qrot_inv(q, nb);
            const V3 db = (nlb - nl * dot(nl, nlb)) * inv + nl * gb;
            clb = mk(k.x != cl.x ? db.x : 0.0f, k.y != cl.y ? db.y : 0.0f, k.z != cl.z ? db.z : 0.0f);
        } else {   // the face hit_box chose; the normal is constant, gap = +-cl_axis - half - r
            float best = hx - cl.x;
            int face = 0;
            if (hx + cl.x < best) { best = hx + cl.x; face = 1; }
            if (hy - cl.y < best) { best = hy - cl.y; face = 2; }
            if (hy + cl.y < best) { best = hy + cl.y; face = 3; }
            if (hz - cl.z < best) { best = hz - cl.z; face = 4; }
            if (hz + cl.z < best) { best = hz + cl.z; face = 5; }
            const float g = (face & 1) ? -gb : gb;
            clb = mk(face >> 1 == 0 ? g : 0.0f, face >> 1 == 1 ? g : 0.0f, face >> 1 == 2 ? g : 0.0f);
        }
        return qrot(q, clb);
    }
    const V3 ca = (x - xyz(A0)) + cr;
    const V3 d = xyz(__ldg(L0 + l * kLinkStride + 1));
    const float tr = dot(ca, d) * (1.0f / sc.link_len);
    const float t = fminf(fmaxf(tr, 0.0f), 1.0f);
    const V3 diff = ca - d * (t * sc.link_len);
    const float d2 = dot(diff, diff);
    if (d2 < 1e-18f) return mk(0, 0, 0);   // centre on the axis: constant normal and gap
    const float inv = rsqrtf(d2);
    const V3 n = diff * inv;
    V3 db = (nb - n * dot(n, nb)) * inv + n * gb;
    if (tr > 0.0f && tr < 1.0f) db = db - d * dot(d, db);   // t follows the centre inside the segment
    return db;
}

__device__ __forceinline__ void outer_add(float (&M)[9], V3 a, V3 b, float s) {
    const float av[3] = {a.x * s, a.y * s, a.z * s}, bv[3] = {b.x, b.y, b.z};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] += av[i] * bv[j];
}

// Reverse of one contact's setup and narrowphase (its record rc: r, gap; n,
// 1/k_n; c, 1/k_t; link, sphere) given the derivatives w.r.t. its constants
// nb, rb, cb, iknb, iktb: the thread's parts of d/dx, d/d(1/m), d/dW and d/dR
// accumulate.
__device__ __forceinline__ void contact_setup_bwd(const float4 *rc, V3 nb, V3 rb, V3 cb, float iknb, float iktb,
                                                  const S6 &Wi, float trW, const M3 &R, V3 x, int sfirst,
                                                  const DevScene &sc, const DevConfig &cfg, const float4 *L0,
                                                  const float4 *L1, float inv_h, float (&Wbar)[9], float (&Rbar)[9],
                                                  V3 &xb_l, float &invm_l) {
    const float4 r0 = rc[0], r1 = rc[1], r2 = rc[2], r3 = rc[3];
    const V3 r = xyz(r0), n = xyz(r1);
    const float gap = r0.w, ikn = r1.w, ikt = r2.w;
    const int l = rec_link(r3), j = __float_as_int(r3.z);
    // 1/k_n and 1/k_t = 2 / (tr K - k_n)
    float knb = -iknb * ikn * ikn;
    const float Db = -iktb * ikt * ikt * 0.5f;
    const float trKb = Db;
    knb -= Db;
    // k_n = 1/m + (r x n) . W (r x n)
    const V3 rn = cross(r, n);
    const V3 rnb = smul(Wi, rn) * (2.0f * knb);
    invm_l += knb + 3.0f * trKb;
    outer_add(Wbar, rn, rn, knb);
    rb = rb + cross(n, rnb);
    nb = nb + cross(rnb, r);
    // tr K = 3/m + |r|^2 tr W - r . W r
    rb = rb + (r * (2.0f * trW) - smul(Wi, r) * 2.0f) * trKb;
    const float rr = dot(r, r) * trKb;
    Wbar[0] += rr; Wbar[4] += rr; Wbar[8] += rr;
    outer_add(Wbar, r, r, -trKb);
    // c = v_link - n b(gap)
    const float bias = contact_bias(cfg, gap);
    const float gb = -dot(n, cb) * bias_slope(cfg, gap);
    nb = nb - cb * bias;
    if (l != 0) {   // v_link = (T_end T_start^-1 p - p) / h, p = x + r
        const float4 Aq = __ldg(L0 + l * kLinkStride + 2), Bq = __ldg(L1 + l * kLinkStride + 2);
        const Q4 qa = {Aq.x, Aq.y, Aq.z, Aq.w}, qe = {Bq.x, Bq.y, Bq.z, Bq.w};
        const V3 yb = (qrot(qa, qrot_inv(qe, cb)) - cb) * inv_h;
        xb_l = xb_l + yb;
        rb = rb + yb;
    }
    // r = R s_j - n r_j, gap and n from the sphere centre x + R s_j
    const float4 s4 = __ldg(sc.spheres + sfirst + j);
    nb = nb - rb * s4.w;
    const V3 cr = mmul(R, xyz(s4));
    const V3 hb = hit_bwd(sc, l, x, cr, L0, gb, nb);
    xb_l = xb_l + hb;
    outer_add(Rbar, rb + hb, xyz(s4), 1.0f);
}

// Reverse of one contact's update in a Jacobi iteration (update_contact with
// constants r, n, c, 1/k_n, 1/k_t against the velocities Vi, Wv, from its
// impulse l0 before the iteration): lb holds the derivative w.r.t. its impulse
// after the iteration and leaves with the one before it; nb, rb, cb, iknb,
// iktb, mu_b and the group's velocity and moment sums acc accumulate.
__device__ __forceinline__ void contact_update_bwd(V3 r, V3 n, V3 cc, float ikn, float ikt, V3 l0, V3 Vi, V3 Wv,
                                                   float mu, float inv_nc, float width, float beta_s, V3 &lb,
                                                   V3 &nb, V3 &rb, V3 &cb, float &iknb, float &iktb, float &mu_b,
                                                   float (&acc)[6]) {
    const V3 u = Vi + cross(Wv, r) - cc;
    const float un = dot(u, n), lo = dot(l0, n);
    const float zn = lo - un * ikn;
    const float ln = fmaxf(zn, 0.0f);
    const V3 ut = u - n * un;
    const V3 zt = (l0 - n * lo) - ut * ikt;
    const float L = mu * ln;
    // lambda' = lambda + (n ln + lt - lambda) / n_c
    const V3 lpb = lb * inv_nc;
    lb = lb * (1.0f - inv_nc);
    float lnb = dot(n, lpb);
    nb = nb + lpb * ln;
    V3 ztb;
    float Lb;
    disk_bwd(zt, L, lpb, width, ztb, Lb);
    lnb += mu * Lb;
    mu_b += ln * Lb;
    const float znb = lnb * sigmoid(beta_s * zn);
    float lob = znb;
    float unb = -znb * ikn;
    iknb -= znb * un;
    // zt = (l0 - n lo) - (u - n un) ikt
    const float nzt = dot(n, ztb);
    lb = lb + ztb;
    nb = nb - ztb * lo;
    lob -= nzt;
    V3 ub = ztb * (-ikt);
    nb = nb + ztb * (ikt * un);
    unb += ikt * nzt;
    iktb -= dot(ut, ztb);
    // lo = l0 . n, un = u . n
    lb = lb + n * lob;
    nb = nb + l0 * lob;
    ub = ub + n * unb;
    nb = nb + u * unb;
    // u = V + W x r - c
    const V3 rxu = cross(r, ub);
    acc[0] += ub.x; acc[1] += ub.y; acc[2] += ub.z;
    acc[3] += rxu.x; acc[4] += rxu.y; acc[5] += rxu.z;
    rb = rb + cross(ub, Wv);
    cb = cb - ub;
}

// Reverse sweep of one substep from start state b (whose forward has just
// been recomputed with a tape; nc contacts). On entry `ad` holds the
// derivatives w.r.t. the substep's end state, on return those w.r.t. b.
// invm_b (lane-uniform) and mu_b (per lane) accumulate d/d(1/m) and d/dmu.
// Not inlined: both tape modes then run the same compiled reverse, so their
// gradients agree bit for bit.
template <int GW, int PL>
__device__ __noinline__ void rev_substep(const AdjArgs &a, const Env &E_, const Body &b_, const float4 *L0,
                                        const float4 *L1, int nc, const SlotPtr &sp_, GroupSm<GW> &S,
                                        const AGroup<GW> &G_, int &parity_, Adj &ad_, float &invm_b_, float &mu_b_) {
    constexpr int T = AGroup<GW>::T;
    // by-value copies (see fwd_substep), written back on return
    const Env E = E_;
    const Body b = b_;
    const SlotPtr sp = sp_;
    const AGroup<GW> G = G_;
    int parity = parity_;
    Adj ad = ad_;
    float invm_b = invm_b_, mu_b = mu_b_;
    const float width = a.width, beta_s = a.beta_s;
    const DevScene sc = a.sc;   // by value, as E below
    const DevConfig cfg = a.cfg;
    const int cap = cfg.c_max, I = E.iters;
    const float h = cfg.h, inv_h = 1.0f / h;
    const V3 grav = mk(cfg.gx * h, cfg.gy * h, cfg.gz * h);
    const V3 v_pred = b.v + grav;
    const V3 w_pred = b.w;
    const M3 R = qmat(b.q);
    const S6 Wi = world_inv_inertia(R, E.Jb, E.inv_m);
    const float trW = Wi.xx + Wi.yy + Wi.zz;
    const bool solved = nc > 0 && I > 0;
    V3 Vf = v_pred, Wf = w_pred;   // body velocity after the solve
    if (solved) {
        const float *s = sp.sh + 8 * (I - 1);
        Vf = v_pred + mk(s[0], s[1], s[2]) * E.inv_m;
        Wf = w_pred + smul(Wi, mk(s[3], s[4], s[5]));
    }

    // -- integration: x' = x + h V, q' = normalize(exp(h W) q)
    V3 Vb = ad.v + ad.x * h;
    V3 Wb = ad.w;
    Q4 qb;
    {
        const float wn = sqrtf(dot(Wf, Wf));
        float sn, cs;
        sincosf(0.5f * wn * h, &sn, &cs);
        const float kq = (wn > 0.0f) ? sn / wn : 0.5f * h;
        const Q4 e = {cs, Wf.x * kq, Wf.y * kq, Wf.z * kq};
        const Q4 p = qmul(e, b.q);
        const float s = rsqrtf(p.w * p.w + p.x * p.x + p.y * p.y + p.z * p.z);
        const Q4 qn = {p.w * s, p.x * s, p.y * s, p.z * s};
        const float dq = ad.q.w * qn.w + ad.q.x * qn.x + ad.q.y * qn.y + ad.q.z * qn.z;
        const Q4 pb = {(ad.q.w - qn.w * dq) * s, (ad.q.x - qn.x * dq) * s, (ad.q.y - qn.y * dq) * s,
                       (ad.q.z - qn.z * dq) * s};
        qb = qmul(qconj(e), pb);                // p = e q: dq = L(e)^T dp
        const Q4 eb = qmul(pb, qconj(b.q));     // de = R(q)^T dp
        // e = (cos(th/2), s(th) A), A = h W, th = |A|, s(th) = sin(th/2) / th
        const float th = wn * h;
        const float sf = kq / h;
        float ds;   // s'(th) / th
        if (th < 0.25f) {
            const float t2 = th * th;
            ds = -1.0f / 24.0f + t2 * (1.0f / 960.0f - t2 * (1.0f / 107520.0f));
        } else {
            ds = (0.5f * th * cs - sn) / (th * th * th);
        }
        const V3 av = Wf * h;
        const V3 ev = mk(eb.x, eb.y, eb.z);
        const V3 ab = av * (-0.5f * sf * eb.w) + ev * sf + av * (ds * dot(av, ev));
        Wb = Wb + ab * h;
    }
    V3 vpb = mk(0, 0, 0), wpb = mk(0, 0, 0);
    float Wbar[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // d/dW, this lane's part
    float Rbar[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // d/dR, this lane's part
    V3 xb_l = mk(0, 0, 0);
    float invm_l = 0.0f;
    if (solved) {
        const float inv_nc = 1.0f / (float)nc;
        V3 lb[PL], nb[PL], rb[PL], cb[PL];
        float iknb[PL], iktb[PL];
        // the contacts' constants in registers, and the tape one iteration ahead:
        // l1_ the impulse after iteration it, l0_ after it - 1 (zero before the
        // first), sc_/sp_ the sums after it and it - 1
        V3 r_[PL], n_[PL], c_[PL], l1_[PL], l0_[PL];
        float ikn_[PL], ikt_[PL];
        auto lam_at = [&](int it, int ci) -> V3 { return it >= 0 ? xyz(sp.lamh[(size_t)it * cap + ci]) : mk(0, 0, 0); };
        auto sums_at = [&](int it, float4 &lo, float4 &hi) {
            if (it >= 0) {
                const float4 *q = reinterpret_cast<const float4 *>(sp.sh + 8 * it);
                lo = q[0]; hi = q[1];
            } else {
                lo = hi = make_float4(0, 0, 0, 0);
            }
        };
#pragma unroll
        for (int k = 0; k < PL; ++k) {
            lb[k] = nb[k] = rb[k] = cb[k] = mk(0, 0, 0);
            iknb[k] = iktb[k] = 0.0f;
            r_[k] = n_[k] = c_[k] = l1_[k] = l0_[k] = mk(0, 0, 0);
            ikn_[k] = ikt_[k] = 0.0f;
            const int ci = G.gt + T * k;
            if (ci < nc) {
                const float4 *rc = sp.rec + 4 * ci;
                const float4 r0 = rc[0], r1 = rc[1], r2 = rc[2], r3 = rc[3];
                r_[k] = xyz(r0); n_[k] = xyz(r1); c_[k] = xyz(r2); ikn_[k] = r1.w; ikt_[k] = r2.w;
                l1_[k] = lam_at(I - 1, ci);
                l0_[k] = lam_at(I - 2, ci);
                const int pad = rec_pad(r3);
                if (pad < sc.n_pads) lb[k] = mk(-S.fbar[3 * pad], -S.fbar[3 * pad + 1], -S.fbar[3 * pad + 2]);
            }
        }
        // contacts past the register slots: their reverse state in sp.adjs
        for (int ci = G.gt + T * PL; ci < nc; ci += T) {
            const int pad = rec_pad(sp.rec[4 * ci + 3]);
            float4 *A = sp.adjs + 4 * ci;
            A[0] = (pad < sc.n_pads) ? make_float4(-S.fbar[3 * pad], -S.fbar[3 * pad + 1], -S.fbar[3 * pad + 2], 0.0f)
                                     : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            A[1] = A[2] = A[3] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        float4 sc_lo, sc_hi, sp_lo, sp_hi;
        sums_at(I - 1, sc_lo, sc_hi);
        sums_at(I - 2, sp_lo, sp_hi);
        for (int it = I - 1; it >= 0; --it) {
            // the tape of iteration it - 2, for the next step, requested now
            V3 pf_[PL];
#pragma unroll
            for (int k = 0; k < PL; ++k) {
                const int ci = G.gt + T * k;
                pf_[k] = (ci < nc) ? lam_at(it - 2, ci) : mk(0, 0, 0);
            }
            float4 pf_lo, pf_hi;
            sums_at(it - 2, pf_lo, pf_hi);
            // (a) V^{it+1} = v_pred + S1 / m, W^{it+1} = w_pred + W S2, sums of the impulses after it
            const V3 S1 = mk(sc_lo.x, sc_lo.y, sc_lo.z), S2 = mk(sc_lo.w, sc_hi.x, sc_hi.y);
            vpb = vpb + Vb;
            wpb = wpb + Wb;
            if (G.gt == 0) {
                invm_l += dot(Vb, S1);
                outer_add(Wbar, Wb, S2, 1.0f);
            }
            const V3 g = smul(Wi, Wb);
            const V3 vm = Vb * E.inv_m;
            // every register slot without a branch (an empty slot has r = l1 = 0
            // and keeps lb = 0, so its reverse below adds zeros)
#pragma unroll
            for (int k = 0; k < PL; ++k) {
                const V3 lbk = lb[k] + vm + cross(g, r_[k]);
                lb[k] = (G.gt + T * k < nc) ? lbk : lb[k];
                rb[k] = rb[k] + cross(l1_[k], g);
            }
            // (b) the contact updates of iteration it, against V^it, W^it
            V3 Vi = v_pred, Wv = w_pred;
            if (it > 0) {
                Vi = v_pred + mk(sp_lo.x, sp_lo.y, sp_lo.z) * E.inv_m;
                Wv = w_pred + smul(Wi, mk(sp_lo.w, sp_hi.x, sp_hi.y));
            }
            float acc[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int k = 0; k < PL; ++k)
                contact_update_bwd(r_[k], n_[k], c_[k], ikn_[k], ikt_[k], l0_[k], Vi, Wv, E.mu, inv_nc, width, beta_s,
                                   lb[k], nb[k], rb[k], cb[k], iknb[k], iktb[k], mu_b, acc);
            for (int ci = G.gt + T * PL; ci < nc; ci += T) {   // (a) and (b) of the contacts in memory
                const float4 *rc = sp.rec + 4 * ci;
                const float4 r0 = rc[0], r1 = rc[1], r2 = rc[2];
                float4 *A = sp.adjs + 4 * ci;
                const float4 a0 = A[0], a1 = A[1], a2 = A[2], a3 = A[3];
                const V3 r = xyz(r0);
                V3 lbk = xyz(a0) + vm + cross(g, r), nbk = xyz(a1), rbk = xyz(a2) + cross(lam_at(it, ci), g),
                   cbk = xyz(a3);
                float iknbk = a0.w, iktbk = a1.w;
                contact_update_bwd(r, xyz(r1), xyz(r2), r1.w, r2.w, lam_at(it - 1, ci), Vi, Wv, E.mu, inv_nc, width,
                                   beta_s, lbk, nbk, rbk, cbk, iknbk, iktbk, mu_b, acc);
                A[0] = make_float4(lbk.x, lbk.y, lbk.z, iknbk);
                A[1] = make_float4(nbk.x, nbk.y, nbk.z, iktbk);
                A[2] = make_float4(rbk.x, rbk.y, rbk.z, 0.0f);
                A[3] = make_float4(cbk.x, cbk.y, cbk.z, 0.0f);
            }
            gsum6<GW>(acc, G, S, parity);
            Vb = mk(acc[0], acc[1], acc[2]);
            Wb = mk(acc[3], acc[4], acc[5]);
#pragma unroll
            for (int k = 0; k < PL; ++k) {
                l1_[k] = l0_[k];
                l0_[k] = pf_[k];
            }
            sc_lo = sp_lo; sc_hi = sp_hi;
            sp_lo = pf_lo; sp_hi = pf_hi;
        }
        vpb = vpb + Vb;   // V^0 = v_pred, W^0 = w_pred
        wpb = wpb + Wb;

        // contact setup and narrowphase, in reverse
#pragma unroll
        for (int k = 0; k < PL; ++k) {
            const int ci = G.gt + T * k;
            if (ci < nc) {
                contact_setup_bwd(sp.rec + 4 * ci, nb[k], rb[k], cb[k], iknb[k], iktb[k], Wi, trW, R, b.x, E.sfirst, sc,
                                  cfg, L0, L1, inv_h, Wbar, Rbar, xb_l, invm_l);
            }
        }
        for (int ci = G.gt + T * PL; ci < nc; ci += T) {
            const float4 *A = sp.adjs + 4 * ci;
            const float4 a0 = A[0], a1 = A[1], a2 = A[2], a3 = A[3];
            contact_setup_bwd(sp.rec + 4 * ci, xyz(a1), xyz(a2), xyz(a3), a0.w, a1.w, Wi, trW, R, b.x, E.sfirst, sc, cfg,
                              L0, L1, inv_h, Wbar, Rbar, xb_l, invm_l);
        }
    } else {
        vpb = vpb + Vb;
        wpb = wpb + Wb;
    }

    // sum the lanes' parts: x (3), 1/m (1), W (9), R (9)
    float r1[6] = {xb_l.x, xb_l.y, xb_l.z, invm_l, Wbar[0], Wbar[1]};
    float r2[6] = {Wbar[2], Wbar[3], Wbar[4], Wbar[5], Wbar[6], Wbar[7]};
    float r3[6] = {Wbar[8], Rbar[0], Rbar[1], Rbar[2], Rbar[3], Rbar[4]};
    float r4[6] = {Rbar[5], Rbar[6], Rbar[7], Rbar[8], 0.0f, 0.0f};
    gsum6<GW>(r1, G, S, parity);
    gsum6<GW>(r2, G, S, parity);
    gsum6<GW>(r3, G, S, parity);
    gsum6<GW>(r4, G, S, parity);
    const float Wt[9] = {r1[4], r1[5], r2[0], r2[1], r2[2], r2[3], r2[4], r2[5], r3[0]};
    float Rt[9] = {r3[1], r3[2], r3[3], r3[4], r3[5], r4[0], r4[1], r4[2], r4[3]};
    // W = R J R^T / m:  d/d(1/m) += <Wbar, R J R^T>,  Rbar += (Wbar + Wbar^T) R J / m
    {
        const float Rm[9] = {R.c0.x, R.c1.x, R.c2.x, R.c0.y, R.c1.y, R.c2.y, R.c0.z, R.c1.z, R.c2.z};
        const float J[9] = {E.Jb.xx, E.Jb.xy, E.Jb.xz, E.Jb.xy, E.Jb.yy, E.Jb.yz, E.Jb.xz, E.Jb.yz, E.Jb.zz};
        float RJ[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) RJ[3 * i + j] = Rm[3 * i] * J[j] + Rm[3 * i + 1] * J[3 + j] + Rm[3 * i + 2] * J[6 + j];
        float inner = 0.0f;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float Mij = RJ[3 * i] * Rm[3 * j] + RJ[3 * i + 1] * Rm[3 * j + 1] + RJ[3 * i + 2] * Rm[3 * j + 2];
                inner += Wt[3 * i + j] * Mij;
            }
        invm_b += r1[3] + inner;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float sacc = 0.0f;
#pragma unroll
                for (int k = 0; k < 3; ++k) sacc += (Wt[3 * i + k] + Wt[3 * k + i]) * RJ[3 * k + j];
                Rt[3 * i + j] += sacc * E.inv_m;
            }
    }
    // R(q) -> q (the polynomial map of qmat)
    {
        const Q4 q = b.q;
        const float R00 = Rt[0], R01 = Rt[1], R02 = Rt[2], R10 = Rt[3], R11 = Rt[4], R12 = Rt[5], R20 = Rt[6],
                    R21 = Rt[7], R22 = Rt[8];
        qb.w += 2.0f * (q.z * (R10 - R01) + q.y * (R02 - R20) + q.x * (R21 - R12));
        qb.x += 2.0f * (-2.0f * q.x * (R11 + R22) + q.y * (R10 + R01) + q.z * (R20 + R02) + q.w * (R21 - R12));
        qb.y += 2.0f * (-2.0f * q.y * (R00 + R22) + q.x * (R10 + R01) + q.z * (R21 + R12) + q.w * (R02 - R20));
        qb.z += 2.0f * (-2.0f * q.z * (R00 + R11) + q.x * (R20 + R02) + q.y * (R21 + R12) + q.w * (R10 - R01));
    }
    ad.x = ad.x + mk(r1[0], r1[1], r1[2]);
    ad.q = qb;
    ad.v = vpb;
    ad.w = wpb;
    ad_ = ad;
    parity_ = parity;
    invm_b_ = invm_b;
    mu_b_ = mu_b;
}

// The refinement step of elite i, taken by the thread that wrote its trial's
// cost (the group's first) at the end of the trial's adjoint launch. The trial
// is accepted when it lowers the elite's cost (the first evaluation always
// is); otherwise the step multiplier halves. Then the next trial steps from
// the best state along the normalised steepest descent in coordinates scaled
// by eta:
//   s = eta * g,  dz = -scale * eta * s / |s|
// (position += dz_0..2, R <- exp([dz_3..5]x) R, m += dz_6, mu += dz_7, with m
// and mu clamped), or, after the last trial, the best state is restored and
// an improved elite's live end state, parameters and window cost (sum and
// mean) replace the scored ones. Not inlined: one copy for the kernel's three
// exits keeps it out of the adjoint's own code.
__device__ __noinline__ void refine_step(const RefineArgs &r, int i) {
    const int env = r.elite[i];
    const double c = r.cost[i];
    const float4 *tp = r.step == 0 ? r.ws_pose : r.tr_pose;
    const float2 *tq = r.step == 0 ? r.ws_params : r.tr_params;
    if (r.step == 0 || c < r.best_c[i]) {
        r.accepted[i] = (r.step == 0 ? 0ull : r.accepted[i]) | (1ull << r.step);
        r.best_pose[2 * i] = tp[2 * env];
        r.best_pose[2 * i + 1] = tp[2 * env + 1];
        for (int q = 0; q < 2; ++q) {
            r.best_end_pose[2 * i + q] = r.end_pose[2 * i + q];
            r.best_end_vel[2 * i + q] = r.end_vel[2 * i + q];
        }
        r.best_params[i] = tq[env];
        for (int d = 0; d < 8; ++d) r.best_grad[8 * i + d] = r.grad[8 * i + d];
        r.best_c[i] = c;
        if (r.step == 0) { r.c0[i] = c; r.scale[i] = 1.0f; }
    } else {
        r.scale[i] *= 0.5f;
    }
    const float4 p0 = r.best_pose[2 * i], p1 = r.best_pose[2 * i + 1];
    float2 th = r.best_params[i];
    if (r.last) {
        r.tr_pose[2 * env] = p0;
        r.tr_pose[2 * env + 1] = p1;
        r.tr_params[env] = th;
        const double cb = r.best_c[i];
        if (cb < r.c0[i]) {   // improved: its best trial's window replaces the scored one
            r.pose[2 * env] = r.best_end_pose[2 * i];
            r.pose[2 * env + 1] = r.best_end_pose[2 * i + 1];
            r.vel[2 * env] = r.best_end_vel[2 * i];
            r.vel[2 * env + 1] = r.best_end_vel[2 * i + 1];
            r.params[env] = th;
            const int nw = *r.n_window;
            r.c_sum[env] = cb;
            r.c_mean[env] = nw > 0 ? cb / (double)nw : cb;
        }
        return;
    }
    float sv[8], nrm2 = 0.0f;
    for (int d = 0; d < 8; ++d) {
        sv[d] = r.eta[d] * r.best_grad[8 * i + d];
        nrm2 += sv[d] * sv[d];
    }
    float dz[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (nrm2 > 0.0f && isfinite(nrm2)) {
        const float f = -r.scale[i] * rsqrtf(nrm2);
        for (int d = 0; d < 8; ++d) dz[d] = f * r.eta[d] * sv[d];
    }
    const float an = sqrtf(dz[3] * dz[3] + dz[4] * dz[4] + dz[5] * dz[5]);
    float sn, cs;
    sincosf(0.5f * an, &sn, &cs);
    const float kq = an > 0.0f ? sn / an : 0.5f;
    const Q4 e = {cs, dz[3] * kq, dz[4] * kq, dz[5] * kq};
    const Q4 q = qnorm(qmul(e, Q4{p1.x, p1.y, p1.z, p1.w}));
    th.x = fminf(fmaxf(th.x + dz[6], r.m_lo), r.m_hi);
    th.y = fminf(fmaxf(th.y + dz[7], r.mu_lo), r.mu_hi);
    r.tr_pose[2 * env] = make_float4(p0.x + dz[0], p0.y + dz[1], p0.z + dz[2], 0.0f);
    r.tr_pose[2 * env + 1] = make_float4(q.w, q.x, q.y, q.z);
    r.tr_params[env] = th;
}

template <int GW, int PL>
__global__ void __launch_bounds__(kABlock) adjoint_kernel(const AdjArgs a) {
    constexpr int T = AGroup<GW>::T, GPB = kAW / GW;
    __shared__ GroupSm<GW> sm[GPB];
    __shared__ PadTab PT;
    const AGroup<GW> G;
    const int lane = G.gt;   // the group's thread (0 .. 32 GW - 1)
    const int slot = blockIdx.x * GPB + G.gid;
    if (threadIdx.x < 32) {   // the pads of each link, in pad order
        int c = 0;
        for (int p = 0; p < a.sc.n_pads && c < kAPadsPerLink; ++p)
            if (__ldg(a.sc.pad_link + p) == (int)threadIdx.x) PT.id[threadIdx.x * kAPadsPerLink + c++] = (unsigned char)p;
        PT.cnt[threadIdx.x] = (unsigned char)c;
    }
    for (int p = threadIdx.x; p < a.sc.n_pads; p += kABlock) {
        PT.s0[p] = __ldg(a.sc.pad_s0 + p);
        PT.s1[p] = __ldg(a.sc.pad_s1 + p);
    }
    __syncthreads();
    if (slot >= a.n) return;   // whole groups only
    GroupSm<GW> &S = sm[G.gid];
    int parity = 0;   // the group's reduction buffer
    const DevScene &sc = a.sc;
    const DevConfig &cfg = a.cfg;
    const int ns = cfg.substeps, Lk = sc.n_links, P = sc.n_pads, cap = cfg.c_max;
    const int env = a.envs ? a.envs[slot] : slot;
    if (env < 0 || env >= a.N) {   // not an environment of the handle
        if (lane < 8) a.grad[8 * slot + lane] = 0.0f;
        if (a.grad_quat && lane < 4) a.grad_quat[4 * slot + lane] = 0.0f;
        if (lane == 0 && a.cost) a.cost[slot] = NAN;
        return;
    }
    const bool seg_tape = a.seg_tape != 0;   // every substep of a segment keeps its tape
    const int nck = (a.H + a.K - 1) / a.K;
    // with whole-segment tapes, the segments recomputed later keep their
    // substeps' contact records from the first pass, and their recomputation
    // replays them
    const int nrec = seg_tape ? (nck - 1) * a.K * ns : 0;
    const SlotLayout Ly = slot_layout(a.H, a.K, ns, P, cap, a.iters_max, seg_tape ? a.K * ns : 1, nrec);
    float *base = a.scratch + (size_t)slot * a.stride;
    SlotPtr sp0;
    sp0.ck = reinterpret_cast<float4 *>(base + Ly.ck);
    sp0.sg = reinterpret_cast<float4 *>(base + Ly.sg);
    sp0.sf = base + Ly.sf;
    sp0.lamf = reinterpret_cast<float4 *>(base + Ly.lamf);
    sp0.adjs = reinterpret_cast<float4 *>(base + Ly.adj);
    sp0.recs = reinterpret_cast<float4 *>(base + Ly.recs);
    sp0.nrc = reinterpret_cast<int *>(base + Ly.nrc);
    sp0.ncs = reinterpret_cast<int *>(base + Ly.ncs);
    sp0.tape = base + Ly.tape;
    sp0.blk_lamh = Ly.blk_lamh;
    sp0.blk_sh = Ly.blk_sh;
    sp0.blk_stride = Ly.blk_stride;
    const SlotPtr sp = sp0.blk(0);

    const float4 P0 = a.pose[2 * env], P1 = a.pose[2 * env + 1];
    const float4 V0 = a.vel[2 * env], V1 = a.vel[2 * env + 1];
    const float2 th = a.params[env];
    const int shp = a.shape[env];
    Env E;
    E.sfirst = __ldg(sc.shape_first + shp);
    E.NS = __ldg(sc.shape_count + shp);
    E.iters = a.iters[env];
    E.mu = th.y;
    E.inv_m = 1.0f / th.x;
    E.bound = __ldg(sc.shape_bound + shp);
    E.cfirst = __ldg(sc.cl_first + shp);
    E.Jb.xx = __ldg(sc.shape_jinv + 6 * shp + 0); E.Jb.yy = __ldg(sc.shape_jinv + 6 * shp + 1);
    E.Jb.zz = __ldg(sc.shape_jinv + 6 * shp + 2); E.Jb.xy = __ldg(sc.shape_jinv + 6 * shp + 3);
    E.Jb.xz = __ldg(sc.shape_jinv + 6 * shp + 4); E.Jb.yz = __ldg(sc.shape_jinv + 6 * shp + 5);
    const Body b0 = {xyz(P0), Q4{P1.x, P1.y, P1.z, P1.w}, xyz(V0), xyz(V1)};
    int st = a.status[env];
    if (E.iters > a.iters_max) st |= IH_ENV_INVALID;   // the tape cannot hold its iterations

    const float h = cfg.h, inv_h = 1.0f / h, inv_ns = 1.0f / (float)ns;
    const size_t tab_frame = (size_t)(ns + 1) * Lk * kLinkStride;
    const float4 *tab0 = a.link_tab + (size_t)a.frame0 * tab_frame;

    // -- pass 1: the cost, the state at every K-th frame, every frame's pad
    //    forces, the substep states of the last segment (the first one
    //    reversed) and its tape, and the contact records of the others
    const int f_last = (nck - 1) * a.K;
    double cost = 0.0;
    Body b = b0;
    for (int f = 0; f < a.H && !(st & kDiverged); ++f) {
        if (f % a.K == 0 && lane == 0) store_body(sp.ck + 4 * (f / a.K), b);
        for (int k = lane; k < 3 * P; k += T) S.padacc[k] = 0.0f;
        G.sync();
        const float4 *tab = tab0 + (size_t)f * tab_frame;
        for (int s = 0; s < ns; ++s) {
            const float4 *L0 = tab + (size_t)s * Lk * kLinkStride;
            if (f >= f_last) {
                const int blk = (f - f_last) * ns + s;
                if (lane == 0) store_body(sp.sg + 4 * blk, b);
                if (seg_tape && !a.forward_only) {   // the last segment's tape, recorded on the way
                    const int nc = fwd_substep<GW, PL>(a, E, b, L0, L0 + Lk * kLinkStride, sp.blk(blk), S, PT, G, parity,
                                                       st, 1 | a.zero, 1 | a.zero, -1);
                    if (lane == 0) sp.ncs[blk] = nc;
                    continue;
                }
            }
            if (nrec > 0 && f < f_last) {   // a segment recomputed later: keep this substep's records
                const int q = f * ns + s;
                SlotPtr sq = sp;
                sq.rec = sp.recs + (size_t)q * cap * 4;
                const int nc = fwd_substep<GW, PL>(a, E, b, L0, L0 + Lk * kLinkStride, sq, S, PT, G, parity, st, a.zero,
                                                   1 | a.zero, -1);
                if (lane == 0) sp.nrc[q] = nc;
                continue;
            }
            fwd_substep<GW, PL>(a, E, b, L0, L0 + Lk * kLinkStride, sp, S, PT, G, parity, st, a.zero, 1 | a.zero, -1);
        }
        for (int k = lane; k < 3 * P; k += T) sp.sf[(size_t)f * 3 * P + k] = S.padacc[k] * inv_ns;
        if (!all_finite(b.x, b.q, b.v, b.w)) st |= IH_ENV_NONFINITE;
        else if (dot(b.x, b.x) > cfg.escape_radius * cfg.escape_radius) st |= IH_ENV_ESCAPED;
        {   // frame cost in FP64, as the scored step: each pad's terms in parallel, summed in pad order
            const float *o = a.obs + (size_t)f * P * 3;
            const double tau = (double)cfg.tau, tau2 = __dmul_rn(tau, tau), wf = (double)cfg.w_force;
            for (int p = lane; p < P; p += T) {
                const double fx = S.padacc[3 * p] * inv_ns, fy = S.padacc[3 * p + 1] * inv_ns,
                             fz = S.padacc[3 * p + 2] * inv_ns;
                const double ox = o[3 * p], oy = o[3 * p + 1], oz = o[3 * p + 2];
                const double dx = __dsub_rn(fx, ox), dy = __dsub_rn(fy, oy), dz = __dsub_rn(fz, oz);
                const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                S.term[p] = __dmul_rn(wf, d2);
                const double n2 = __dadd_rn(__dadd_rn(__dmul_rn(fx, fx), __dmul_rn(fy, fy)), __dmul_rn(fz, fz));
                const double no = __dadd_rn(__dadd_rn(__dmul_rn(ox, ox), __dmul_rn(oy, oy)), __dmul_rn(oz, oz));
                S.flag[p] = (n2 > tau2) != (no > tau2);
            }
            G.sync();
            if (lane == 0) {
                double cf = 0.0;
                for (int p = 0; p < P; ++p) {
                    cf = __dadd_rn(cf, S.term[p]);
                    if (S.flag[p]) cf = __dadd_rn(cf, (double)cfg.w_contact);
                }
                cost = __dadd_rn(cost, cf);
            }
        }
        G.sync();
    }
    if (a.out_pose && lane == 0) {   // the horizon's end state (not meaningful when diverged)
        a.out_pose[2 * slot] = make_float4(b.x.x, b.x.y, b.x.z, 0.0f);
        a.out_pose[2 * slot + 1] = make_float4(b.q.w, b.q.x, b.q.y, b.q.z);
        a.out_vel[2 * slot] = make_float4(b.v.x, b.v.y, b.v.z, 0.0f);
        a.out_vel[2 * slot + 1] = make_float4(b.w.x, b.w.y, b.w.z, 0.0f);
    }
    if (a.forward_only) {
        if (lane == 0 && a.cost) a.cost[slot] = (st & kDiverged) ? INFINITY : cost;
        if (lane == 0 && a.refine) refine_step(a.rf, slot);
        return;
    }
    if (st & kDiverged) {   // no derivative of a diverged or invalid environment
        if (lane < 8) a.grad[8 * slot + lane] = 0.0f;
        if (a.grad_quat && lane < 4) a.grad_quat[4 * slot + lane] = 0.0f;
        if (lane == 0 && a.cost) a.cost[slot] = INFINITY;
        __syncwarp();   // (the refinement step reads the whole gradient)
        if (lane == 0 && a.refine) refine_step(a.rf, slot);
        return;
    }

    // -- pass 2: segments in reverse
    Adj ad = {mk(0, 0, 0), Q4{0, 0, 0, 0}, mk(0, 0, 0), mk(0, 0, 0)};
    float invm_b = 0.0f, mu_b = 0.0f;
    const float wf2 = 2.0f * cfg.w_force * inv_h * inv_ns;
    for (int seg = nck - 1; seg >= 0; --seg) {
        const int fb = seg * a.K, fe = min(a.H, fb + a.K);
        b = load_body(sp.ck + 4 * seg);
        // the segment's substep start states and tapes (its frames' pad forces
        // are the first pass's)
        for (int f = fb; f < fe && seg < nck - 1; ++f) {
            const float4 *tab = tab0 + (size_t)f * tab_frame;
            for (int s = 0; s < ns; ++s) {
                const int blk = (f - fb) * ns + s;
                if (lane == 0) store_body(sp.sg + 4 * blk, b);
                const float4 *L0 = tab + (size_t)s * Lk * kLinkStride;
                if (seg_tape) {   // replaying the first pass's records of the substep
                    const int q = f * ns + s;
                    SlotPtr sq = sp.blk(blk);
                    sq.rec = sp.recs + (size_t)q * cap * 4;
                    const int nc = fwd_substep<GW, PL>(a, E, b, L0, L0 + Lk * kLinkStride, sq, S, PT, G, parity, st,
                                                       1 | a.zero, a.zero, sp.nrc[q]);
                    if (lane == 0) sp.ncs[blk] = nc;
                } else {
                    fwd_substep<GW, PL>(a, E, b, L0, L0 + Lk * kLinkStride, sp, S, PT, G, parity, st, a.zero, a.zero,
                                        -1);
                }
            }
        }
        for (int f = fe - 1; f >= fb; --f) {
            const float *o = a.obs + (size_t)f * P * 3;
            for (int k = lane; k < 3 * P; k += T)
                S.fbar[k] = wf2 * (sp.sf[(size_t)f * 3 * P + k] - o[k]);
            G.sync();
            const float4 *tab = tab0 + (size_t)f * tab_frame;
            for (int s = ns - 1; s >= 0; --s) {
                const float4 *L0 = tab + (size_t)s * Lk * kLinkStride;
                const float4 *L1 = L0 + Lk * kLinkStride;
                const int blk = (f - fb) * ns + s;
                const Body bs = load_body(sp.sg + 4 * blk);
                if (seg_tape) {
                    G.sync();
                    SlotPtr sq = sp.blk(blk);
                    if (seg < nck - 1) sq.rec = sp.recs + (size_t)(f * ns + s) * cap * 4;   // (the replayed records)
                    rev_substep<GW, PL>(a, E, bs, L0, L1, sp.ncs[blk], sq, S, G, parity, ad, invm_b, mu_b);
                } else {   // re-run the substep once more, recording its tape
                    Body bt = bs;
                    int st2 = 0;
                    const int nc = fwd_substep<GW, PL>(a, E, bt, L0, L1, sp, S, PT, G, parity, st2, 1 | a.zero, a.zero, -1);
                    rev_substep<GW, PL>(a, E, bs, L0, L1, nc, sp, S, G, parity, ad, invm_b, mu_b);
                }
            }
            G.sync();
        }
    }
    {
        float mv[6] = {mu_b, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        gsum6<GW>(mv, G, S, parity);
        mu_b = mv[0];
    }
    if (lane == 0) {
        // rotation tangent: q = exp(delta) q0, d/d delta at 0 = vec(qbar (x) conj(q0)) / 2
        const Q4 g = qmul(ad.q, qconj(b0.q));
        float *gr = a.grad + 8 * slot;
        gr[0] = ad.x.x; gr[1] = ad.x.y; gr[2] = ad.x.z;
        gr[3] = 0.5f * g.x; gr[4] = 0.5f * g.y; gr[5] = 0.5f * g.z;
        gr[6] = -invm_b * E.inv_m * E.inv_m;
        gr[7] = mu_b;
        if (a.grad_quat) {
            a.grad_quat[4 * slot + 0] = ad.q.w; a.grad_quat[4 * slot + 1] = ad.q.x;
            a.grad_quat[4 * slot + 2] = ad.q.y; a.grad_quat[4 * slot + 3] = ad.q.z;
        }
        if (a.cost) a.cost[slot] = cost;
        if (a.refine) refine_step(a.rf, slot);
    }
}

template <int GW, int PL>
cudaError_t launch_pl(const AdjArgs &a, cudaStream_t s) {
    constexpr int GPB = kAW / GW;
    adjoint_kernel<GW, PL><<<(a.n + GPB - 1) / GPB, kABlock, 0, s>>>(a);
    return cudaGetLastError();
}

__global__ void iters_max_kernel(int n, int N, const int *envs, const int *iters, int *out) {
    int m = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int e = envs ? envs[i] : i;
        if (e >= 0 && e < N) m = max(m, iters[e]);
    }
    m = __reduce_max_sync(kFull, m);
    __shared__ int part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, part[w]);
        *out = m;
    }
}

}  // namespace

size_t adjoint_scratch_floats(int H, int K, int substeps, int n_pads, int c_max, int iters_max, bool seg_tape) {
    const int nck = (H + K - 1) / K;
    return slot_layout(H, K, substeps, n_pads, c_max, iters_max, seg_tape ? K * substeps : 1,
                       seg_tape ? (nck - 1) * K * substeps : 0).total;
}

cudaError_t launch_adjoint_iters_max(int n, int N, const int *envs, const int *iters, int *out, cudaStream_t s) {
    iters_max_kernel<<<1, 256, 0, s>>>(n, N, envs, iters, out);
    return cudaGetLastError();
}

#ifndef IH_ADJ_GROUPS_PER_SM
#define IH_ADJ_GROUPS_PER_SM 2
#endif
bool adjoint_variant_supported(int gw, int pl) {
    return (gw == 0 && pl == 0) || (gw == 4 && pl == 1) || (gw == 1 && (pl == 1 || pl == 2));
}

// Automatic shape. Few environments (the refined elites, a small batch), at
// most two per SM -- the blocks of ~250 registers a thread that an SM holds:
// four warps each, so that their contacts' chains run side by side, one
// contact a thread in registers. More: one warp each (no barriers between the
// warps of an environment) with one contact a thread in registers when no
// shape has more than 32 spheres (a substep's contacts then rarely exceed a
// warp: 22 at most for the 27-sphere box), else two (the 64-sphere cylinder
// reaches ~100); four a thread spilled and ran slower. Contacts beyond the
// register slots run from scratch memory.
cudaError_t launch_adjoint(const AdjArgs &a, cudaStream_t s) {
    if (a.gw == 4 && a.pl == 1) return launch_pl<4, 1>(a, s);
    if (a.gw == 1 && a.pl == 1) return launch_pl<1, 1>(a, s);
    if (a.gw == 1 && a.pl == 2) return launch_pl<1, 2>(a, s);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (a.n <= IH_ADJ_GROUPS_PER_SM * sms) return launch_pl<4, 1>(a, s);
    if (a.s_max <= 32) return launch_pl<1, 1>(a, s);
    return launch_pl<1, 2>(a, s);
}

}  // namespace ih
