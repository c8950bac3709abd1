// full_cost.cuh -- the full cost of Sec. III-C over the PD hand's observation,
// in FP64, used by the per-frame cost kernel and by the frames' cost launches
// of a PD window (cost.cu). Every operation is an explicitly rounded FP64
// intrinsic, so both compute the same bits in the same order:
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

// atan2(|a x b|, a . b)
__device__ __forceinline__ double fc_angle(double ax, double ay, double az, double bx, double by, double bz) {
    const double cx = __dsub_rn(__dmul_rn(ay, bz), __dmul_rn(az, by));
    const double cy = __dsub_rn(__dmul_rn(az, bx), __dmul_rn(ax, bz));
    const double cz = __dsub_rn(__dmul_rn(ax, by), __dmul_rn(ay, bx));
    return atan2(sqrt(fc_dot3(cx, cy, cz, cx, cy, cz)), fc_dot3(ax, ay, az, bx, by, bz));
}

// w1 |q - q_gt|
__device__ __forceinline__ double full_cost_joints(const float *q, const float *g, int D, double w1) {
    double dq = 0.0;
    for (int j = 0; j < D; ++j) {
        const double d = __dsub_rn((double)q[j], (double)g[j]);
        dq = __dadd_rn(dq, __dmul_rn(d, d));
    }
    return __dmul_rn(w1, sqrt(dq));
}

// the terms of one pad: positions and rotations (x y z, 0 | w x y z), forces,
// slip records (d_x, d_y, flag bits, 0), of the environment (a) and the truth (b)
__device__ __forceinline__ double full_cost_pad(const double (&w)[10], double tau, float4 pa, float4 qa, float4 pb,
                                                float4 qb, const float *fa, const float *fb, float4 sa, float4 sb) {
    const double dx = __dsub_rn((double)pa.x, (double)pb.x), dy = __dsub_rn((double)pa.y, (double)pb.y),
                 dz = __dsub_rn((double)pa.z, (double)pb.z);
    double c = __dmul_rn(w[1], sqrt(fc_dot3(dx, dy, dz, dx, dy, dz)));
    // R_a^-1 R_b: conj(qa) qb
    const double aw = qa.x, ax = -(double)qa.y, ay = -(double)qa.z, az = -(double)qa.w;
    const double bw = qb.x, bx = qb.y, by = qb.z, bz = qb.w;
    const double rw = __dsub_rn(__dsub_rn(__dsub_rn(__dmul_rn(aw, bw), __dmul_rn(ax, bx)), __dmul_rn(ay, by)), __dmul_rn(az, bz));
    const double rx = __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(aw, bx), __dmul_rn(ax, bw)), __dmul_rn(ay, bz)), __dmul_rn(az, by));
    const double ry = __dadd_rn(__dadd_rn(__dsub_rn(__dmul_rn(aw, by), __dmul_rn(ax, bz)), __dmul_rn(ay, bw)), __dmul_rn(az, bx));
    const double rz = __dadd_rn(__dsub_rn(__dadd_rn(__dmul_rn(aw, bz), __dmul_rn(ax, by)), __dmul_rn(ay, bx)), __dmul_rn(az, bw));
    c = __dadd_rn(c, __dmul_rn(w[2], __dmul_rn(2.0, atan2(sqrt(fc_dot3(rx, ry, rz, rx, ry, rz)), fabs(rw)))));
    const double fax = fa[0], fay = fa[1], faz = fa[2], fbx = fb[0], fby = fb[1], fbz = fb[2];
    const double ma = sqrt(fc_dot3(fax, fay, faz, fax, fay, faz)), mb = sqrt(fc_dot3(fbx, fby, fbz, fbx, fby, fbz));
    const bool in_a = ma > tau, in_b = mb > tau;
    if (in_a != in_b) {
        c = __dadd_rn(c, w[3]);
    } else {
        c = __dadd_rn(c, __dmul_rn(w[4], fabs(__dsub_rn(ma, mb))));
        if (in_a) c = __dadd_rn(c, __dmul_rn(w[5], fc_angle(fax, fay, faz, fbx, fby, fbz)));
    }
    const int ga = __float_as_int(sa.z), gb = __float_as_int(sb.z);
    const int ta = ga & 1, tb = gb & 1;
    if (ta != tb) {
        c = __dadd_rn(c, w[6]);
    } else if (ta) {
        const double d0 = sa.x, d1 = sa.y, e0 = sb.x, e1 = sb.y;
        const double cr = fabs(__dsub_rn(__dmul_rn(d0, e1), __dmul_rn(d1, e0)));
        c = __dadd_rn(c, __dmul_rn(w[7], atan2(cr, __dadd_rn(__dmul_rn(d0, e0), __dmul_rn(d1, e1)))));
    }
    const int ra = (ga >> 1) & 1, rb = (gb >> 1) & 1;
    if (ra != rb) {
        c = __dadd_rn(c, w[8]);
    } else if (ra) {
        c = __dadd_rn(c, __dmul_rn(w[9], fabs((double)((ga >> 2) & 1) - (double)((gb >> 2) & 1))));
    }
    return c;
}

}  // namespace ih
