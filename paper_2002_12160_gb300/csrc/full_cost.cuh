// full_cost.cuh -- the full cost of Sec. III-C over the PD hand's observation,
// in FP64, shared by the cost kernel (cost.cu) and the PD step's window mode
// (step_pd.cu). Every operation is an explicitly rounded FP64 intrinsic, so
// both translation units compute the same bits in the same order (the cost
// kernel one environment per thread; the PD window one pad quantity per lane,
// four lanes per pad, the pad sums and the total then in the same order):
//   cost = w1 |q - q_gt| + sum over pads, in pad order, of
//          w2 |P - P_gt| + w3 angle(R^-1 R_gt)
//          + w4 (1 - alpha) + alpha (w5 | |c| - |c_gt| | + w6 angle(c, c_gt))
//          + w7 (1 - beta) + beta w8 angle(d, d_gt) + w9 (1 - gamma) + gamma w10 |r - r_gt|
// with the force angle only when both pads are in contact, the slip angle only
// when both slip and |r - r_gt| only when both slip rotationally.
#pragma once

#include "internal.cuh"

namespace ih {

__device__ __forceinline__ double fc_dot3(double ax, double ay, double az, double bx, double by, double bz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(ax, bx), __dmul_rn(ay, by)), __dmul_rn(az, bz));
}

// w1 |q - q_gt|: the squared differences summed in joint order
__device__ __forceinline__ double full_cost_joints(const float *q, const float *g, int D, double w1) {
    double dq = 0.0;
    for (int j = 0; j < D; ++j) {
        const double d = __dsub_rn((double)q[j], (double)g[j]);
        dq = __dadd_rn(dq, __dmul_rn(d, d));
    }
    return __dmul_rn(w1, sqrt(dq));
}

// One of a pad's four measured quantities, k = 0..3, every k by the same
// instructions (so that four lanes of a warp can take one pad's four without
// diverging). On the pair of 4-vectors (a0, a), (b0, b) it forms
//   s = a0 b0 + a . b,  v = a0 b - b0 a - a x b
// (for unit quaternions A, B: conj(A) B = (s, v)) and returns
//   k = 0: the rotation angle of R_a^-1 R_b, 2 atan2(|v|, |s|), A = q_a, B = q_b
//   k = 1: the force angle atan2(|c_a x c_b|, c_a . c_b), A = (0, c_a), B = (0, c_b)
//   k = 2: the slip angle, the same on (0, d_a, 0), (0, d_b, 0)
//   k = 3: the distance |P_a - P_b|, A = (1, 0), B = (0, P_a - P_b)
// and in na, nb the lengths |a|, |b| (for k = 1 the two force magnitudes).
// Pad poses are (x y z, 0 | w x y z), slip records (d_x, d_y, flag bits, 0).
__device__ __forceinline__ double fc_pad_term(int k, float4 pa, float4 qa, float4 pb, float4 qb, const float *fa,
                                              const float *fb, float4 sa, float4 sb, double &na, double &nb) {
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f, b0 = 0.0f, b1 = 0.0f, b2 = 0.0f, b3 = 0.0f;
    float c1 = 0.0f, c2 = 0.0f, c3 = 0.0f;   // subtracted from (b1, b2, b3) in FP64
    if (k == 0) {
        a0 = qa.x; a1 = qa.y; a2 = qa.z; a3 = qa.w;
        b0 = qb.x; b1 = qb.y; b2 = qb.z; b3 = qb.w;
    } else if (k == 1) {
        a1 = fa[0]; a2 = fa[1]; a3 = fa[2];
        b1 = fb[0]; b2 = fb[1]; b3 = fb[2];
    } else if (k == 2) {
        a1 = sa.x; a2 = sa.y;
        b1 = sb.x; b2 = sb.y;
    } else {
        a0 = 1.0f;
        b1 = pa.x; b2 = pa.y; b3 = pa.z;
        c1 = pb.x; c2 = pb.y; c3 = pb.z;
    }
    const double A0 = a0, A1 = a1, A2 = a2, A3 = a3, B0 = b0;
    const double B1 = __dsub_rn((double)b1, (double)c1), B2 = __dsub_rn((double)b2, (double)c2),
                 B3 = __dsub_rn((double)b3, (double)c3);
    const double s = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(A0, B0), __dmul_rn(A1, B1)), __dmul_rn(A2, B2)),
                               __dmul_rn(A3, B3));
    const double vx = __dsub_rn(__dsub_rn(__dmul_rn(A0, B1), __dmul_rn(B0, A1)),
                                __dsub_rn(__dmul_rn(A2, B3), __dmul_rn(A3, B2)));
    const double vy = __dsub_rn(__dsub_rn(__dmul_rn(A0, B2), __dmul_rn(B0, A2)),
                                __dsub_rn(__dmul_rn(A3, B1), __dmul_rn(A1, B3)));
    const double vz = __dsub_rn(__dsub_rn(__dmul_rn(A0, B3), __dmul_rn(B0, A3)),
                                __dsub_rn(__dmul_rn(A1, B2), __dmul_rn(A2, B1)));
    const double y = sqrt(fc_dot3(vx, vy, vz, vx, vy, vz));
    na = sqrt(fc_dot3(A1, A2, A3, A1, A2, A3));
    nb = sqrt(fc_dot3(B1, B2, B3, B1, B2, B3));
    const double ang = __dmul_rn(k == 0 ? 2.0 : 1.0, atan2(y, k == 0 ? fabs(s) : s));
    return k == 3 ? y : ang;
}

// A pad's cost terms from its four quantities t[k] (fc_pad_term) and force
// magnitudes ma, mb, added in the order
//   w2 |P - P_gt| + w3 angle(R^-1 R_gt) + [w4 (1 - alpha) + alpha w5 | |c| - |c_gt| |]
//   + alpha w6 angle(c, c_gt) + [w7 (1 - beta) + beta w8 angle(d, d_gt)]
//   + [w9 (1 - gamma) + gamma w10 |r - r_gt|]
// (a bracket is one addition; alpha: both pads or neither in contact, the
// force angle only when both are; beta, gamma likewise for slip and rotational
// slip). Every product is formed and the unused ones selected away, so the
// lanes of a warp do not diverge; adding 0.0 leaves the non-negative sum as is.
__device__ __forceinline__ double fc_pad_combine(const double (&w)[10], double tau, const double *t, double ma,
                                                 double mb, float sa_z, float sb_z) {
    const bool in_a = ma > tau, in_b = mb > tau;
    const int ga = __float_as_int(sa_z), gb = __float_as_int(sb_z);
    const int ta = ga & 1, tb = gb & 1, ra = (ga >> 1) & 1, rb = (gb >> 1) & 1;
    const double pf = __dmul_rn(w[4], fabs(__dsub_rn(ma, mb))), pc = __dmul_rn(w[5], t[1]);
    const double ps = __dmul_rn(w[7], t[2]);
    const double pr = __dmul_rn(w[9], fabs((double)((ga >> 2) & 1) - (double)((gb >> 2) & 1)));
    double c = __dmul_rn(w[1], t[3]);
    c = __dadd_rn(c, __dmul_rn(w[2], t[0]));
    c = __dadd_rn(c, in_a != in_b ? w[3] : pf);
    c = __dadd_rn(c, in_a && in_b ? pc : 0.0);
    c = __dadd_rn(c, ta != tb ? w[6] : (ta ? ps : 0.0));
    c = __dadd_rn(c, ra != rb ? w[8] : (ra ? pr : 0.0));
    return c;
}

// |c| of a force in FP64 (the same operations as fc_pad_term's na, nb for k = 1)
__device__ __forceinline__ double fc_len(const float *c) {
    const double x = c[0], y = c[1], z = c[2];
    return sqrt(fc_dot3(x, y, z, x, y, z));
}

// The terms of one pad of the environment (a) against the truth (b), one
// thread: its quantities in turn, then their sum. The force and slip angles
// are formed only when fc_pad_combine selects them (both pads in contact,
// both slipping); otherwise it adds a constant or nothing, so the sum has the
// bits of the four-lane form, which forms every quantity.
__device__ __forceinline__ double full_cost_pad(const double (&w)[10], double tau, float4 pa, float4 qa, float4 pb,
                                                float4 qb, const float *fa, const float *fb, float4 sa, float4 sb) {
    double t[4] = {0.0, 0.0, 0.0, 0.0}, na, nb;
    t[0] = fc_pad_term(0, pa, qa, pb, qb, fa, fb, sa, sb, na, nb);
    t[3] = fc_pad_term(3, pa, qa, pb, qb, fa, fb, sa, sb, na, nb);
    const double ma = fc_len(fa), mb = fc_len(fb);
    if (ma > tau && mb > tau) t[1] = fc_pad_term(1, pa, qa, pb, qb, fa, fb, sa, sb, na, nb);
    if ((__float_as_int(sa.z) & 1) && (__float_as_int(sb.z) & 1)) t[2] = fc_pad_term(2, pa, qa, pb, qb, fa, fb, sa, sb, na, nb);
    return fc_pad_combine(w, tau, t, ma, mb, sa.z, sb.z);
}

}  // namespace ih
