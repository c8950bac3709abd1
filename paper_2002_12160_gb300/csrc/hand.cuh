// hand.cuh -- forward kinematics of one finger (a serial chain of four
// revolute joints), shared by the commanded-trajectory table (setup.cu) and
// the PD-driven hand's per-environment step (step_pd.cu).
#pragma once

#include "internal.cuh"

namespace ih {

// Quaternion chain of finger f for joint angles qf[0..3]:
//   Q_0 = qz(yaw + q_0) qy(-pi/2),  a_0 = root,
//   a_j = a_{j-1} + L Q_{j-1} e_x,  Q_j = Q_{j-1} qy(-q_j).
// Writes per link (a, 0), (Q e_x, 0), (Q as w x y z) to out[4][kLinkStride].
// With zax/org non-null also the joints: joint 0 turns about +z through the
// root, joint j >= 1 by -q_j about link j's y axis through a_j, so its axis
// (for positive q_j) is -Q_j e_y.
__device__ __forceinline__ void finger_fk(const DevScene &sc, int f, const float (&qf)[4], float4 *out,
                                          float4 *zax = nullptr, float4 *org = nullptr) {
    const float4 root = sc.finger_root[f];
    float sz, cz, sy, cy;
    sincosf(0.5f * (root.w + qf[0]), &sz, &cz);
    const float hs = 0.70710678118654752f;   // sin(pi/4) = cos(pi/4)
    // qz(yaw + q0) * qy(-pi/2)
    Q4 Q = qmul({cz, 0.0f, 0.0f, sz}, {hs, 0.0f, -hs, 0.0f});
    V3 a = mk(root.x, root.y, root.z);
    for (int j = 0; j < 4; ++j) {
        if (j > 0) {
            a = a + qrot(Q, mk(sc.link_len, 0, 0));
            sincosf(-0.5f * qf[j], &sy, &cy);
            Q = qnorm(qmul(Q, {cy, 0.0f, sy, 0.0f}));
        }
        const V3 ax = qrot(Q, mk(1, 0, 0));
        float4 *lo = out + j * kLinkStride;
        lo[0] = make_float4(a.x, a.y, a.z, 0.0f);
        lo[1] = make_float4(ax.x, ax.y, ax.z, 0.0f);
        lo[2] = make_float4(Q.w, Q.x, Q.y, Q.z);
        if (zax) {
            const V3 z = (j == 0) ? mk(0, 0, 1) : qrot(Q, mk(0, -1, 0));
            zax[j] = make_float4(z.x, z.y, z.z, 0.0f);
            org[j] = make_float4(a.x, a.y, a.z, 0.0f);
        }
    }
}

}  // namespace ih
