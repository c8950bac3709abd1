// step_pd.cu -- the dynamics step with a PD-driven articulated hand: the
// hand's joint angles are part of each environment's state (Sec. III-A, s_t
// holds the joint angles of articulated bodies) and follow the desired joint
// positions u_t through a joint-angle PD controller (Sec. IV), pushed back by
// the contacts. Each environment also reports the full observation o_t: the
// joint angles q_t, every pad's pose (P_t, R_t), its force c_t, and its
// translational slip direction d_t and rotational slip r_t (Sec. III-A).
//
// One warp owns one environment at a time (grid-stride, LPT order). Per
// substep the warp
//   1. runs the fingers' kinematics from the environment's own joint angles
//      (one lane per finger) into shared memory, with every joint's axis and
//      origin, and predicts the joints' velocities under the PD force alone:
//      qd* = (I qd + h kp (u - q)) / M, M = I + h kd + h^2 kp (implicit PD);
//   2. culls links against the object's bounding sphere, then (link, 8-sphere
//      cluster) pairs by the clusters' enclosing spheres, tests the spheres of
//      the surviving pairs and compacts contacts in pair order;
//   3. sets each contact up: effective masses gain the joints' share
//      sum_a (J_a . n)^2 / M, J_a = z_a x (p - o_a) over the joints that move
//      the contact's link;
//   4. runs the Jacobi iterations on the object and the joints together (the
//      first 96 contacts held in registers, three per lane): each
//      contact updates against the object velocity and its link's velocity
//      (link twist w_l x p + c_l from the joints), the warp sums the object's
//      impulse and moment, the lane of each joint sums the impulses of the
//      link it ends at and their moments about the origin, a suffix over the
//      finger's lanes gives it qd_a = qd*_a - z_a . sum_{links moved by a}
//      (T_l - o_a x F_l) / M, and a prefix over them the links' new twists;
//   5. integrates the object and the joints (q += h qd), and adds each
//      contact's impulse to its pad, with the impulse-weighted relative slip
//      velocity, normal and spin for the slip sensing.
// At the end of a frame the fingers' kinematics at the final joint angles give
// the pads' poses, and the slip sums give d_t and r_t. A window launch (T
// frames) writes every frame's observation, status and pose; the frames' full
// cost and window means are then formed by launches of their own (cost.cu),
// so this kernel does no FP64 work.
#include <cstddef>

#include "contact.cuh"
#include "hand.cuh"
#include "internal.cuh"

namespace ih {
namespace {

constexpr int kPdBlock = 128;                 // four environments per block
constexpr int kPdWarps = kPdBlock / 32;
constexpr int kPdMaxLinks = 1 + 4 * IH_MAX_FINGERS;
constexpr int kPdMaxJoints = 4 * IH_MAX_FINGERS;
constexpr int kPdPadsPerLink = 4;
constexpr int kPdSlots = 3;                   // register-resident contacts per lane

// per-warp (per-environment) records
struct PdWarp {
    float4 link[kPdMaxLinks][kLinkStride];    // link poses: (a, 0), (axis, 0), (quat)
    float4 zax[kPdMaxJoints], org[kPdMaxJoints];
    float4 tw[kPdMaxLinks][2];                // link twist: w_l, c_l (v(p) = w_l x p + c_l)
    float qd_star[kPdMaxJoints], qd[kPdMaxJoints], qj[kPdMaxJoints];
    float padf[3 * IH_MAX_PADS];              // force sums over the frame's substeps
    float slip[8 * IH_MAX_PADS];              // per pad: w, w vt (3), w n (3), w spin
    unsigned short lbeg[kPdMaxLinks], lend[kPdMaxLinks];
    unsigned char links[kPdMaxLinks];
    int pad_;
    float4 clc[IH_MAX_SPHERES / kCluster];    // cluster centres (world-rotated, relative to x), radius
    unsigned short clp[kPdMaxLinks * (IH_MAX_SPHERES / kCluster)];   // surviving (link, cluster) pairs
    float4 opp[IH_MAX_PADS][2];               // the frame's pad poses: (position, 0), (quaternion)
    float4 osl[IH_MAX_PADS];                  // the frame's slip records: (d_x, d_y, flag bits, 0)
    double pterm[IH_MAX_PADS];                // window mode: each pad's cost terms
};
static_assert(sizeof(PdWarp) % 16 == 0, "warp records keep 16-byte alignment");

__host__ __device__ constexpr size_t pd_align16(size_t b) { return (b + 15) & ~size_t(15); }
// block tables: pads per link and their axial intervals
__host__ __device__ constexpr size_t pd_block_bytes() {
    return pd_align16(kPdMaxLinks) + pd_align16(kPdMaxLinks * kPdPadsPerLink) + 2 * pd_align16(4 * IH_MAX_PADS);
}
// per warp: the record, then c_max contacts x 4 float4 and s_max spheres
__host__ __device__ inline size_t pd_warp_bytes(int s_max, int c_max) {
    return sizeof(PdWarp) + (4 * (size_t)c_max + (size_t)s_max) * sizeof(float4);
}

// the link's bounding capsule (or the palm box) inflated by the object's
// bound and the margin, from the shared-memory link table
__device__ __forceinline__ bool pd_link_reaches(const DevScene &sc, const DevConfig &cfg, const float4 (*L)[3],
                                                int l, V3 x, float bound) {
    const V3 xa = x - xyz(L[l][0]);
    if (l == 0) {
        const float4 qq = L[0][2];
        const V3 cl = qrot_inv({qq.x, qq.y, qq.z, qq.w}, xa);
        const V3 k3 = mk(fminf(fmaxf(cl.x, -sc.palm_hx), sc.palm_hx), fminf(fmaxf(cl.y, -sc.palm_hy), sc.palm_hy),
                         fminf(fmaxf(cl.z, -sc.palm_hz), sc.palm_hz));
        const V3 dd = cl - k3;
        const float reach = bound + cfg.margin;
        return dot(dd, dd) < reach * reach;
    }
    const V3 ld = xyz(L[l][1]);
    const float t = fminf(fmaxf(dot(xa, ld), 0.0f), sc.link_len);
    const V3 dd = xa - ld * t;
    const float reach = bound + sc.link_rad + cfg.margin;
    return dot(dd, dd) < reach * reach;
}

// the fingers' kinematics at the warp's joint angles W.qj (one lane per finger)
__device__ __forceinline__ void pd_fk(const DevScene &sc, PdWarp &W, int lane) {
    if (lane == 0) {   // palm: identity pose at the origin
        W.link[0][0] = make_float4(0, 0, 0, 0);
        W.link[0][1] = make_float4(1, 0, 0, 0);
        W.link[0][2] = make_float4(1, 0, 0, 0);
    }
    if (lane < sc.n_fingers) {
        const float qf[4] = {W.qj[4 * lane], W.qj[4 * lane + 1], W.qj[4 * lane + 2], W.qj[4 * lane + 3]};
        finger_fk(sc, lane, qf, &W.link[1 + 4 * lane][0], &W.zax[4 * lane], &W.org[4 * lane]);
    }
}

// Every link's twist from the joint velocities, one lane per joint (lane a =
// 4 f + j holds joint j of finger f with velocity qd, axis z = z_a and
// zo = z_a x o_a, kept in registers over a substep's iterations): joint a adds
// (qd z_a, -qd z_a x o_a) to the twist of every link it moves, so the twist of
// link a + 1 is the inclusive prefix over the finger's lanes 4 f .. a (two
// shuffle levels). Every lane of the warp takes part; lanes >= D hold zeros.
__device__ __forceinline__ void pd_joint_twists(PdWarp &W, int lane, int D, V3 z, V3 zo, float qd) {
    V3 wv = z * qd, cv = zo * (-qd);
#pragma unroll
    for (int off = 1; off < 4; off <<= 1) {
        const float a0 = __shfl_up_sync(0xffffffffu, wv.x, off), a1 = __shfl_up_sync(0xffffffffu, wv.y, off),
                    a2 = __shfl_up_sync(0xffffffffu, wv.z, off), b0 = __shfl_up_sync(0xffffffffu, cv.x, off),
                    b1 = __shfl_up_sync(0xffffffffu, cv.y, off), b2 = __shfl_up_sync(0xffffffffu, cv.z, off);
        if ((lane & 3) >= off) {
            wv = wv + mk(a0, a1, a2);
            cv = cv + mk(b0, b1, b2);
        }
    }
    if (lane < D) {
        W.tw[lane + 1][0] = make_float4(wv.x, wv.y, wv.z, 0.0f);
        W.tw[lane + 1][1] = make_float4(cv.x, cv.y, cv.z, 0.0f);
    }
}

// (a budget of two blocks per SM: the register-resident contacts need it)
__global__ void __launch_bounds__(kPdBlock, 2) pd_step_kernel(const PdArgs a, int s_max) {
    extern __shared__ __align__(16) unsigned char smem[];
    const DevScene &sc = a.sc;
    const DevConfig &cfg = a.cfg;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int ns = cfg.substeps, Lk = sc.n_links, P = sc.n_pads, D = sc.n_joints;
    const float h = cfg.h, inv_h = 1.0f / h, inv_L = 1.0f / sc.link_len;
    const V3 grav = mk(cfg.gx * h, cfg.gy * h, cfg.gz * h);
    const float Mj = cfg.armature + h * cfg.kd + h * h * cfg.kp, inv_Mj = 1.0f / Mj;
    const int cap = cfg.c_max;
    const float inv_ns = 1.0f / (float)ns;
    // window mode (pose_frames != null): every frame's observation written out
    // for the frames' cost launches, the argmin taken afterwards
    const bool window_mode = a.pose_frames != nullptr;

    unsigned char *pl_cnt = smem;
    unsigned char *pl_id = smem + pd_align16(kPdMaxLinks);
    float *p_s0 = reinterpret_cast<float *>(smem + pd_align16(kPdMaxLinks) + pd_align16(kPdMaxLinks * kPdPadsPerLink));
    float *p_s1 = p_s0 + IH_MAX_PADS;
    unsigned char *wbase = smem + pd_block_bytes() + wid * pd_warp_bytes(s_max, cap);
    PdWarp &W = *reinterpret_cast<PdWarp *>(wbase);
    // contacts: [0] (r, 0), [1] (n, link | pad << 8 | sphere << 16), [2] (b, 1/k_n, 1/k_t, 0), [3] lambda
    float4 (*stage)[4] = reinterpret_cast<float4 (*)[4]>(wbase + sizeof(PdWarp));
    float4 *sph = &stage[cap][0];

    if (threadIdx.x < kPdMaxLinks) {
        int c = 0;
        for (int p = 0; p < P && c < kPdPadsPerLink; ++p)
            if (__ldg(sc.pad_link + p) == (int)threadIdx.x) pl_id[threadIdx.x * kPdPadsPerLink + c++] = (unsigned char)p;
        pl_cnt[threadIdx.x] = (unsigned char)c;
    }
    for (int p = threadIdx.x; p < P; p += kPdBlock) {
        p_s0[p] = __ldg(sc.pad_s0 + p);
        p_s1[p] = __ldg(sc.pad_s1 + p);
    }
    __syncthreads();

    unsigned long long work[6] = {0, 0, 0, 0, 0, 0};
    for (int slot = blockIdx.x * kPdWarps + wid; slot < a.N; slot += gridDim.x * kPdWarps) {
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
        const int cfirst = __ldg(sc.cl_first + shp);
        for (int k = lane; k < D; k += 32) {
            W.qj[k] = a.qj[(size_t)env * D + k];
            W.qd[k] = a.qdj[(size_t)env * D + k];
        }
        __syncwarp();
        // the observation of the frame just stepped (pad poses from the joints
        // at its end, slip from the frame's sums) into W.opp / W.osl
        auto frame_obs = [&]() {
            pd_fk(sc, W, lane);
            __syncwarp();
            for (int p = lane; p < P; p += 32) {
                const int l = __ldg(sc.pad_link + p);
                const float4 A0 = W.link[l][0], Aq = W.link[l][2];
                const Q4 lq = {Aq.x, Aq.y, Aq.z, Aq.w};
                V3 c;
                if (l == 0) {
                    c = xyz(A0) + qrot(lq, mk(0, 0, sc.palm_hz));
                } else {
                    const float s1 = fminf(p_s1[p], 1.0f), s0 = fmaxf(p_s0[p], 0.0f);
                    c = xyz(A0) + qrot(lq, mk(0.5f * (s0 + s1) * sc.link_len, 0, 0));
                }
                W.opp[p][0] = make_float4(c.x, c.y, c.z, 0.0f);
                W.opp[p][1] = Aq;
                const float *S = W.slip + 8 * p;
                float dx = 0.0f, dy = 0.0f;
                int flags = 0;
                if (S[0] > 0.0f) {
                    const float iw = 1.0f / S[0];
                    const V3 vt = mk(S[1], S[2], S[3]) * iw;
                    V3 nb = mk(S[4], S[5], S[6]);
                    nb = nb * rsqrtf(dot(nb, nb));
                    const float spin = S[7] * iw;
                    if (sqrtf(dot(vt, vt)) > cfg.v_slip) {
                        const V3 ax = xyz(W.link[l][1]);
                        V3 e1 = ax - nb * dot(ax, nb);
                        e1 = e1 * rsqrtf(dot(e1, e1));
                        const V3 e2 = cross(nb, e1);
                        const float d1 = dot(vt, e1), d2 = dot(vt, e2), idn = rsqrtf(d1 * d1 + d2 * d2);
                        dx = d1 * idn;
                        dy = d2 * idn;
                        flags |= 1;
                    }
                    if (fabsf(spin) > cfg.w_slip) flags |= (spin > 0.0f) ? 6 : 2;
                }
                W.osl[p] = make_float4(dx, dy, __int_as_float(flags), 0.0f);
            }
            __syncwarp();
        };

        for (int fr = 0; fr < a.n_frames; ++fr) {
            for (int k = lane; k < 3 * P; k += 32) W.padf[k] = 0.0f;
            for (int k = lane; k < 8 * P; k += 32) W.slip[k] = 0.0f;
            const int frame = a.frame0 + fr;
            const bool skip = (st & kDiverged) != 0;
            for (int s = 0; s < ns && !skip; ++s) {
                // -- 1. the hand at the substep start; the joints under the PD force alone
                pd_fk(sc, W, lane);
                const float frac = (float)(s + 1) / (float)ns;
                for (int k = lane; k < D; k += 32) {
                    const float u0 = __ldg(a.cmd + (size_t)frame * D + k), u1 = __ldg(a.cmd + (size_t)(frame + 1) * D + k);
                    const float u = u0 + frac * (u1 - u0);
                    W.qd_star[k] = (cfg.armature * W.qd[k] + h * cfg.kp * (u - W.qj[k])) * inv_Mj;
                }
                const V3 v_pred = v + grav;
                const V3 w_pred = w;
                const M3 R = qmat(q);
                S6 Jb;
                Jb.xx = __ldg(sc.shape_jinv + 6 * shp + 0); Jb.yy = __ldg(sc.shape_jinv + 6 * shp + 1);
                Jb.zz = __ldg(sc.shape_jinv + 6 * shp + 2); Jb.xy = __ldg(sc.shape_jinv + 6 * shp + 3);
                Jb.xz = __ldg(sc.shape_jinv + 6 * shp + 4); Jb.yz = __ldg(sc.shape_jinv + 6 * shp + 5);
                const S6 Wi = world_inv_inertia(R, Jb, inv_m);
                for (int j = lane; j < NS; j += 32) {
                    const float4 sp = __ldg(sc.spheres + sfirst + j);
                    const V3 cr = mmul(R, xyz(sp));
                    sph[j] = make_float4(cr.x, cr.y, cr.z, sp.w);
                }
                for (int k = lane; k < ncl; k += 32) {
                    const float4 cl = __ldg(sc.clusters + cfirst + k);
                    const V3 cr = mmul(R, xyz(cl));
                    W.clc[k] = make_float4(cr.x, cr.y, cr.z, cl.w);
                }
                __syncwarp();
                for (int k = lane; k < D; k += 32) W.qd[k] = W.qd_star[k];

                // -- 2. cull links, then (surviving link, cluster) pairs by the clusters'
                //       enclosing spheres, then the spheres of the surviving pairs in pair order
                const unsigned ml = __ballot_sync(0xffffffffu, lane < Lk && pd_link_reaches(sc, cfg, W.link, lane, x, bound));
                const int nsurv = __popc(ml);
                if (lane < Lk && ((ml >> lane) & 1u)) W.links[__popc(ml & ((1u << lane) - 1u))] = (unsigned char)lane;
                __syncwarp();
                const int ncp = nsurv * ncl;
                int nclp = 0;
                for (int p0 = 0; p0 < ncp; p0 += 32) {
                    const int p = p0 + lane;
                    bool keep = false;
                    int li = 0, k = 0;
                    if (p < ncp) {
                        li = p / ncl;
                        k = p - li * ncl;
                        const float4 cc = W.clc[k];
                        keep = pd_link_reaches(sc, cfg, W.link, W.links[li], x + xyz(cc), cc.w);
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, keep);
                    if (keep) W.clp[nclp + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)((li << 8) | k);
                    nclp += __popc(bal);
                }
                __syncwarp();
                const int npairs = nclp * kCluster;
                int nc = 0;
                for (int p0 = 0; p0 < npairs; p0 += 32) {
                    const int p = p0 + lane;
                    bool hit = false;
                    Hit hh = {0.0f, mk(0, 0, 1), 0.0f};
                    V3 r = mk(0, 0, 0);
                    int l = 0, j = 0;
                    if (p < npairs) {
                        const int e = W.clp[p / kCluster];
                        j = (e & 0xff) * kCluster + (p % kCluster);
                        l = W.links[e >> 8];
                    }
                    if (p < npairs && j < NS) {   // (j >= NS: padding of the shape's last cluster)
                        const float4 sp = sph[j];
                        const V3 cr = xyz(sp);
                        const float4 A0 = W.link[l][0], Aq = W.link[l][2];
                        const Q4 lq = {Aq.x, Aq.y, Aq.z, Aq.w};
                        if (l == 0) {
                            hh = hit_box(x + cr, sp.w, xyz(A0), lq, sc.palm_hx, sc.palm_hy, sc.palm_hz);
                        } else {
                            hh = hit_capsule((x - xyz(A0)) + cr, sp.w, xyz(W.link[l][1]), sc.link_len, inv_L,
                                             sc.link_rad, lq);
                        }
                        r = cr - hh.n * sp.w;
                        hit = hh.gap < cfg.margin;
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, hit);
                    const int idx = nc + __popc(bal & ((1u << lane) - 1u));
                    if (hit && idx < cap) {
                        int pad = -1;
                        const int npl = pl_cnt[l];
                        for (int k = 0; k < npl; ++k) {
                            const int pp = pl_id[l * kPdPadsPerLink + k];
                            if (l == 0) { pad = pp; break; }
                            const float s0 = p_s0[pp], s1 = p_s1[pp];
                            if (hh.t >= s0 && (hh.t < s1 || s1 >= 1.0f)) { pad = pp; break; }
                        }
                        stage[idx][0] = make_float4(r.x, r.y, r.z, hh.gap);
                        stage[idx][1] = make_float4(hh.n.x, hh.n.y, hh.n.z,
                                                    __int_as_float(l | ((pad & 0xff) << 8) | (j << 16)));
                    }
                    nc += __popc(bal);
                }
                __syncwarp();
                if (nc > cap) {   // more contacts than the per-env capacity
                    st |= IH_ENV_OVERFLOW;
                    nc = 0;
                }
                if (lane == 0) {
                    work[0] += (unsigned long long)npairs;
                    work[5] += (unsigned long long)ncp;
                    work[1] += nc;
                    work[2] += nc > 0 ? (unsigned long long)nc * iters : 0ull;
                    work[3] += 1;
                    work[4] += nc > 0 ? iters : 0;
                }

                // -- 3. contact setup; each link's contact range (empty for links without contacts)
                if (lane < Lk) { W.lbeg[lane] = 0; W.lend[lane] = 0; }
                __syncwarp();
                const float trW = Wi.xx + Wi.yy + Wi.zz;
                for (int ci = lane; ci < nc; ci += 32) {
                    const float4 s0 = stage[ci][0], s1 = stage[ci][1];
                    const int l = __float_as_int(s1.w) & 0xff;
                    if (ci == 0 || (__float_as_int(stage[ci - 1][1].w) & 0xff) != l) W.lbeg[l] = (unsigned short)ci;
                    if (ci == nc - 1 || (__float_as_int(stage[ci + 1][1].w) & 0xff) != l) W.lend[l] = (unsigned short)(ci + 1);
                    const V3 r = xyz(s0), n = xyz(s1);
                    const V3 rn = cross(r, n);
                    float kn = inv_m + dot(rn, smul(Wi, rn));
                    float trK = 3.0f * inv_m + dot(r, r) * trW - dot(r, smul(Wi, r));
                    if (l >= 1) {   // the joints that move the link
                        const int f = (l - 1) >> 2, jl = (l - 1) & 3;
                        const V3 p = x + r;
                        for (int aa = 0; aa <= jl; ++aa) {
                            const int ja = 4 * f + aa;
                            const V3 J = cross(xyz(W.zax[ja]), p - xyz(W.org[ja]));
                            const float jn = dot(J, n);
                            kn += jn * jn * inv_Mj;
                            trK += dot(J, J) * inv_Mj;
                        }
                    }
                    stage[ci][2] = make_float4(contact_bias(cfg, s0.w), 1.0f / kn, 2.0f / (trK - kn), 0.0f);
                    stage[ci][3] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                }
                __syncwarp();

                // -- 4. Jacobi iterations over the object and the joints
                V3 vv = v_pred, ww = w_pred;
                if (nc > 0) {
                    const float inv_nc = 1.0f / (float)nc;
                    // the links' twists under the PD prediction alone (palm: at rest)
                    if (lane == 0) {
                        W.tw[0][0] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        W.tw[0][1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    }
                    // the joint's axis, z_a x o_a and qd*_a stay in registers over the iterations
                    V3 jz = mk(0, 0, 0), jzo = mk(0, 0, 0);
                    float jqs = 0.0f;
                    if (lane < D) {
                        jz = xyz(W.zax[lane]);
                        jzo = cross(jz, xyz(W.org[lane]));
                        jqs = W.qd_star[lane];
                    }
                    pd_joint_twists(W, lane, D, jz, jzo, jqs);
                    __syncwarp();
                    // with at most 16 joints, lanes a and a + 16 split link a + 1's contacts
                    const bool split = D <= 16;
                    const int ja = split ? (lane & 15) : lane, part = split ? (lane >> 4) : 0, stride = split ? 2 : 1;
                    // the first kPdSlots x 32 contacts held in registers over the iterations
                    // (contact ci = lane + 32 k in slot k); an empty slot (link 0 at rest,
                    // r = 0, n = z, bias and 1/k 0, lambda 0) keeps lambda = 0 and adds zeros
                    V3 sr[kPdSlots], sn[kPdSlots], slam[kPdSlots];
                    float sbias[kPdSlots], sikn[kPdSlots], sikt[kPdSlots];
                    int slink[kPdSlots];
#pragma unroll
                    for (int k = 0; k < kPdSlots; ++k) {
                        const int ci = lane + 32 * k;
                        sr[k] = mk(0, 0, 0); sn[k] = mk(0, 0, 1); slam[k] = mk(0, 0, 0);
                        sbias[k] = 0.0f; sikn[k] = 0.0f; sikt[k] = 0.0f; slink[k] = 0;
                        if (ci < nc) {
                            const float4 s0 = stage[ci][0], s1 = stage[ci][1], s2 = stage[ci][2];
                            sr[k] = xyz(s0); sn[k] = xyz(s1); slink[k] = __float_as_int(s1.w) & 0xff;
                            sbias[k] = s2.x; sikn[k] = s2.y; sikt[k] = s2.z;
                        }
                    }
                    for (int it = 0; it < iters; ++it) {
                        float acc[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
                        for (int k = 0; k < kPdSlots; ++k) {
                            if (32 * k < nc) {   // the same for the whole warp
                                const int l = slink[k];
                                const V3 vl = cross(xyz(W.tw[l][0]), x + sr[k]) + xyz(W.tw[l][1]);
                                const V3 cc = vl - sn[k] * sbias[k];
                                slam[k] = update_contact(slam[k], sr[k], sn[k], cc, sikn[k], sikt[k], vv, ww, mu, inv_nc);
                                if (lane + 32 * k < nc)
                                    stage[lane + 32 * k][3] = make_float4(slam[k].x, slam[k].y, slam[k].z, 0.0f);
                                const V3 tq = cross(sr[k], slam[k]);
                                acc[0] += slam[k].x; acc[1] += slam[k].y; acc[2] += slam[k].z;
                                acc[3] += tq.x; acc[4] += tq.y; acc[5] += tq.z;
                            }
                        }
                        for (int ci = 32 * kPdSlots + lane; ci < nc; ci += 32) {
                            const float4 s0 = stage[ci][0], s1 = stage[ci][1], s2 = stage[ci][2], s3 = stage[ci][3];
                            const int l = __float_as_int(s1.w) & 0xff;
                            const V3 r = xyz(s0), n = xyz(s1);
                            const V3 vl = cross(xyz(W.tw[l][0]), x + r) + xyz(W.tw[l][1]);
                            const V3 cc = vl - n * s2.x;
                            const V3 lam = update_contact(xyz(s3), r, n, cc, s2.y, s2.z, vv, ww, mu, inv_nc);
                            stage[ci][3] = make_float4(lam.x, lam.y, lam.z, 0.0f);
                            const V3 tq = cross(r, lam);
                            acc[0] += lam.x; acc[1] += lam.y; acc[2] += lam.z;
                            acc[3] += tq.x; acc[4] += tq.y; acc[5] += tq.z;
                        }
                        __syncwarp();   // this iteration's impulses, for the joints' lanes
                        // lane a = 4 f + j sums the contacts of link a + 1 (its impulses and
                        // their moments about the origin), then a suffix over the finger's
                        // four lanes gives joint a the links it moves, and
                        // qd_a = qd*_a - z_a . sum_{links at or beyond a} (T_l - o_a x F_l) / M
                        float sv[6] = {0, 0, 0, 0, 0, 0};
                        if (ja < D) {
                            const int e = W.lend[ja + 1];
                            for (int ci = W.lbeg[ja + 1] + part; ci < e; ci += stride) {
                                const V3 lam = xyz(stage[ci][3]);
                                const V3 t = cross(x + xyz(stage[ci][0]), lam);
                                sv[0] += lam.x; sv[1] += lam.y; sv[2] += lam.z;
                                sv[3] += t.x; sv[4] += t.y; sv[5] += t.z;
                            }
                        }
                        // the object's sums over the warp and the joints' shares are two
                        // independent chains of shuffles, kept in one straight stretch of code
                        width_sum6<32>(acc, 0xffffffffu, lane);
#pragma unroll
                        for (int k = 0; k < 6; ++k) {
                            const float o = __shfl_down_sync(0xffffffffu, sv[k], 16);
                            sv[k] += split ? o : 0.0f;
                        }
#pragma unroll
                        for (int off = 1; off < 4; off <<= 1) {
                            float o[6];
#pragma unroll
                            for (int k = 0; k < 6; ++k) o[k] = __shfl_down_sync(0xffffffffu, sv[k], off);
                            if ((lane & 3) + off < 4) {
#pragma unroll
                                for (int k = 0; k < 6; ++k) sv[k] += o[k];
                            }
                        }
                        float qd_new = 0.0f;
                        if (lane < D) {
                            const V3 Fs = mk(sv[0], sv[1], sv[2]), Ts = mk(sv[3], sv[4], sv[5]);
                            // z . (T - o x F) = z . T - F . (z x o)
                            const float g = dot(jz, Ts) - dot(Fs, jzo);
                            qd_new = jqs - g * inv_Mj;
                            W.qd[lane] = qd_new;
                        }
                        vv = v_pred + mk(acc[0], acc[1], acc[2]) * inv_m;
                        ww = w_pred + smul(Wi, mk(acc[3], acc[4], acc[5]));
                        pd_joint_twists(W, lane, D, jz, jzo, qd_new);   // for the next iteration and the slip sensing
                        __syncwarp();
                    }
                }
                v = vv;
                w = ww;

                // -- 5. integrate the object and the joints (contact points stay
                //       those of the substep start: p = x_s + r)
                const V3 x_s = x;
                x = x + v * h;
                {
                    const float wn = sqrtf(dot(w, w));
                    float sn, cs;
                    sincosf(0.5f * wn * h, &sn, &cs);
                    const float kq = (wn > 0.0f) ? sn / wn : 0.5f * h;
                    q = qnorm(qmul({cs, w.x * kq, w.y * kq, w.z * kq}, q));
                }
                // (W.tw holds the links' twists at the final joint velocities)
                for (int k = lane; k < D; k += 32) W.qj[k] += h * W.qd[k];
                // pads: force -lambda / h per contact, and the slip sums weighted
                // by the normal impulse
                for (int p = lane; p < P; p += 32) {
                    const int l = __ldg(sc.pad_link + p);
                    float fx = 0.0f, fy = 0.0f, fz = 0.0f;
                    float sw = 0.0f, s1x = 0.0f, s1y = 0.0f, s1z = 0.0f, snx = 0.0f, sny = 0.0f, snz = 0.0f, ssp = 0.0f;
                    const V3 wl = xyz(W.tw[l][0]), cl = xyz(W.tw[l][1]);
                    const int e = W.lend[l];
                    for (int ci = W.lbeg[l]; ci < e; ++ci) {
                        if (((__float_as_int(stage[ci][1].w) >> 8) & 0xff) != p) continue;
                        const V3 lam = xyz(stage[ci][3]), r = xyz(stage[ci][0]), n = xyz(stage[ci][1]);
                        fx -= lam.x * inv_h; fy -= lam.y * inv_h; fz -= lam.z * inv_h;
                        const float ln = dot(lam, n);
                        if (!(ln > 0.0f)) continue;
                        const V3 vrel = (v + cross(w, r)) - (cross(wl, x_s + r) + cl);
                        const V3 vt = vrel - n * dot(vrel, n);
                        const float spin = dot(w - wl, n);
                        sw += ln;
                        s1x += ln * vt.x; s1y += ln * vt.y; s1z += ln * vt.z;
                        snx += ln * n.x; sny += ln * n.y; snz += ln * n.z;
                        ssp += ln * spin;
                    }
                    W.padf[3 * p] += fx; W.padf[3 * p + 1] += fy; W.padf[3 * p + 2] += fz;
                    float *A = W.slip + 8 * p;
                    A[0] += sw; A[1] += s1x; A[2] += s1y; A[3] += s1z; A[4] += snx; A[5] += sny; A[6] += snz; A[7] += ssp;
                }
                __syncwarp();
            }
            if (!skip) {
                bool fin = all_finite(x, q, v, w);
                for (int k = lane; k < D; k += 32) fin = fin && isfinite(W.qj[k]) && isfinite(W.qd[k]);
                fin = __all_sync(0xffffffffu, fin);
                if (!fin) st |= IH_ENV_NONFINITE;
                else if (dot(x, x) > cfg.escape_radius * cfg.escape_radius) st |= IH_ENV_ESCAPED;
            }
            if (window_mode) {   // this frame's observation, status and pose
                frame_obs();
                const size_t ef = (size_t)fr * a.N + env;
                for (int p = lane; p < P; p += 32) {
                    a.fo_pp[2 * (ef * P + p)] = W.opp[p][0];
                    a.fo_pp[2 * (ef * P + p) + 1] = W.opp[p][1];
                    a.fo_slip[ef * P + p] = W.osl[p];
                }
                for (int k = lane; k < 3 * P; k += 32) a.fo_forces[ef * 3 * P + k] = W.padf[k] * inv_ns;
                for (int k = lane; k < D; k += 32) a.fo_q[ef * D + k] = W.qj[k];
                if (lane == 0) {
                    a.fo_status[ef] = st;
                    a.pose_frames[2 * ef] = make_float4(x.x, x.y, x.z, 0.0f);
                    a.pose_frames[2 * ef + 1] = make_float4(q.w, q.x, q.y, q.z);
                }
                __syncwarp();
            }
        }
        // the observation of the last frame: forces, pad poses, slip
        if (!window_mode) frame_obs();
        for (int k = lane; k < 3 * P; k += 32) a.forces[(size_t)env * P * 3 + k] = W.padf[k] * inv_ns;
        for (int p = lane; p < P; p += 32) {
            a.pad_pose[2 * ((size_t)env * P + p)] = W.opp[p][0];
            a.pad_pose[2 * ((size_t)env * P + p) + 1] = W.opp[p][1];
            a.slip[(size_t)env * P + p] = W.osl[p];
        }
        for (int k = lane; k < D; k += 32) {
            a.qj[(size_t)env * D + k] = W.qj[k];
            a.qdj[(size_t)env * D + k] = W.qd[k];
        }
        if (lane == 0) {
            a.pose[2 * env] = make_float4(x.x, x.y, x.z, 0.0f);
            a.pose[2 * env + 1] = make_float4(q.w, q.x, q.y, q.z);
            a.vel[2 * env] = make_float4(v.x, v.y, v.z, 0.0f);
            a.vel[2 * env + 1] = make_float4(w.x, w.y, w.z, 0.0f);
            a.status[env] = st;
        }
        __syncwarp();
    }
    if (lane == 0 && a.work)
        for (int k = 0; k < 6; ++k)
            if (work[k]) atomicAdd(a.work + k, work[k]);
}

// every environment's hand at rest at q0 (D values; null: zero)
__global__ void hand_rest_kernel(int N, int D, const float *q0, float *qj, float *qdj) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)N * D) return;
    qj[k] = q0 ? q0[k % D] : 0.0f;
    qdj[k] = 0.0f;
}

}  // namespace

cudaError_t launch_hand_rest(int N, int D, const float *q0, float *qj, float *qdj, cudaStream_t s) {
    const size_t n = (size_t)N * D;
    if (n == 0) return cudaSuccess;
    hand_rest_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(N, D, q0, qj, qdj);
    return cudaGetLastError();
}

size_t pd_step_smem_bytes(int s_max, int c_max) { return pd_block_bytes() + kPdWarps * pd_warp_bytes(s_max, c_max); }

cudaError_t pd_step_prepare(int s_max, int c_max) {
    const size_t bytes = pd_step_smem_bytes(s_max, c_max);
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(pd_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// one warp per environment, at most four blocks per SM (grid-stride beyond)
int pd_step_grid(int N, int sms) {
    const int need = (N + kPdWarps - 1) / kPdWarps;
    return need < 4 * sms ? need : 4 * sms;
}

cudaError_t launch_pd_step(const PdArgs &a, int grid, int s_max, cudaStream_t s) {
    pd_step_kernel<<<grid, kPdBlock, pd_step_smem_bytes(s_max, a.cfg.c_max), s>>>(a, s_max);
    return cudaGetLastError();
}

}  // namespace ih
