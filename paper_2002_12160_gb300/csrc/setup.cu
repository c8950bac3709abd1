// setup.cu -- kernels that prepare the step: each shape's centroid frame,
// unit inertia and bounding radius; the kinematic hand's link poses for a
// block of commanded frames (the robot state driven by u_t, Sec. III-A); the
// initial sampling of pose, mass and friction (Sec. III-D, Algorithm 1
// initialisation); and the validated upload of a caller's state.
#include "hand.cuh"
#include "internal.cuh"

namespace ih {
namespace {

// One block per shape. Centroid of the sphere centres, recentred spheres,
// unit inertia J = (1/S) sum_s [(2/5) r_s^2 I + |c_s|^2 I - c_s c_s^T] of
// equal solid balls about the centroid, its inverse, and the bounding radius
// max_s |c_s| + r_s.
__global__ void shape_setup_kernel(const float4 *in, float4 *out, const int *first, const int *count,
                                   float *jinv, float *bound, const int *cl_first, float4 *clusters) {
    __shared__ double red[7][256];
    const int sh = blockIdx.x, t = threadIdx.x;
    const int f = first[sh], S = count[sh];
    double cx = 0, cy = 0, cz = 0;
    for (int j = t; j < S; j += blockDim.x) {
        const float4 s = in[f + j];
        cx += s.x; cy += s.y; cz += s.z;
    }
    red[0][t] = cx; red[1][t] = cy; red[2][t] = cz;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) for (int k = 0; k < 3; ++k) red[k][t] += red[k][t + o];
        __syncthreads();
    }
    const double mx = red[0][0] / S, my = red[1][0] / S, mz = red[2][0] / S;
    __syncthreads();
    double a[7] = {0, 0, 0, 0, 0, 0, 0};   // xx yy zz xy xz yz, bound
    for (int j = t; j < S; j += blockDim.x) {
        const float4 s = in[f + j];
        const double x = s.x - mx, y = s.y - my, z = s.z - mz, r = s.w;
        out[f + j] = make_float4((float)x, (float)y, (float)z, s.w);
        const double ball = 0.4 * r * r;
        a[0] += ball + y * y + z * z;
        a[1] += ball + x * x + z * z;
        a[2] += ball + x * x + y * y;
        a[3] -= x * y;
        a[4] -= x * z;
        a[5] -= y * z;
        a[6] = fmax(a[6], sqrt(x * x + y * y + z * z) + r);
    }
    for (int k = 0; k < 7; ++k) red[k][t] = a[k];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) {
            for (int k = 0; k < 6; ++k) red[k][t] += red[k][t + o];
            red[6][t] = fmax(red[6][t], red[6][t + o]);
        }
        __syncthreads();
    }
    if (t == 0) {
        const double xx = red[0][0] / S, yy = red[1][0] / S, zz = red[2][0] / S;
        const double xy = red[3][0] / S, xz = red[4][0] / S, yz = red[5][0] / S;
        // adjugate of the symmetric matrix
        const double c00 = yy * zz - yz * yz, c11 = xx * zz - xz * xz, c22 = xx * yy - xy * xy;
        const double c01 = xz * yz - xy * zz, c02 = xy * yz - xz * yy, c12 = xy * xz - xx * yz;
        const double det = xx * c00 + xy * c01 + xz * c02;
        float *o = jinv + 6 * sh;
        o[0] = (float)(c00 / det); o[1] = (float)(c11 / det); o[2] = (float)(c22 / det);
        o[3] = (float)(c01 / det); o[4] = (float)(c02 / det); o[5] = (float)(c12 / det);
        // rounded outward so that culling with it stays conservative in FP32
        bound[sh] = (float)(red[6][0] * (1.0 + 1e-6)) + 1e-7f;
    }
    // clusters of kCluster consecutive spheres: centre of their centres and the
    // radius that encloses them, in the centroid frame
    const int ncl = (S + kCluster - 1) / kCluster;
    for (int k = t; k < ncl; k += blockDim.x) {
        const int j0 = k * kCluster, j1 = min(S, j0 + kCluster);
        double cx2 = 0, cy2 = 0, cz2 = 0;
        for (int j = j0; j < j1; ++j) {
            const float4 sp = in[f + j];
            cx2 += sp.x - mx; cy2 += sp.y - my; cz2 += sp.z - mz;
        }
        cx2 /= (j1 - j0); cy2 /= (j1 - j0); cz2 /= (j1 - j0);
        double rr = 0;
        for (int j = j0; j < j1; ++j) {
            const float4 sp = in[f + j];
            const double dx = sp.x - mx - cx2, dy = sp.y - my - cy2, dz = sp.z - mz - cz2;
            rr = fmax(rr, sqrt(dx * dx + dy * dy + dz * dz) + sp.w);
        }
        clusters[cl_first[sh] + k] =
            make_float4((float)cx2, (float)cy2, (float)cz2, (float)(rr * (1.0 + 1e-6)) + 1e-7f);
    }
}

// One thread per (substep boundary, finger): quaternion chain of the finger
//   Q_0 = qz(yaw + q_0) qy(-pi/2),  a_0 = root,
//   a_j = a_{j-1} + L Q_{j-1} e_x,  Q_j = Q_{j-1} qy(-q_j).
// Boundary k of frame f uses q = q_f + (k / ns)(q_{f+1} - q_f).
// Output per link: (a, 0), (Q e_x, 0), (Q as w x y z).
__global__ void fk_kernel(const DevScene sc, const float *q, int n_frames, int ns, float4 *tab) {
    const int F = sc.n_fingers, D = sc.n_joints, Lk = sc.n_links;
    const int per = (F > 0) ? F : 1;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n_frames * (ns + 1) * per) return;
    const int b = id / per, f = id % per;
    const int fr = b / (ns + 1), k = b % (ns + 1);
    float4 *o = tab + (size_t)b * Lk * kLinkStride;
    if (f == 0) {   // palm: identity pose at the origin
        o[0] = make_float4(0, 0, 0, 0);
        o[1] = make_float4(1, 0, 0, 0);
        o[2] = make_float4(1, 0, 0, 0);
    }
    if (F == 0) return;
    const float frac = (float)k / (float)ns;
    float qf[4];
    for (int j = 0; j < 4; ++j) {
        const float q0 = q[(size_t)fr * D + 4 * f + j], q1 = q[(size_t)(fr + 1) * D + 4 * f + j];
        qf[j] = q0 + frac * (q1 - q0);
    }
    finger_fk(sc, f, qf, o + (1 + 4 * f) * kLinkStride);
}

// One thread per environment: x = x0 + sigma_p n_{0..2}, R = exp(sigma_r n_{3..5}) R0,
// m, mu uniform; normals from Philox counter (0, 0, i, 0..2), uniforms from block 3.
__global__ void sample_initial_kernel(int N, float4 x0, float4 q0, float sigma_p, float sigma_r,
                                      float m_lo, float m_hi, float mu_lo, float mu_hi,
                                      uint64_t seed, float4 *pose, float4 *vel, float2 *params,
                                      int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double n[6];
    for (int b = 0; b < 3; ++b) gauss2(rng_words(seed, 0, 0, (uint32_t)i, (uint32_t)b), n[2 * b], n[2 * b + 1]);
    const uint4 u = rng_words(seed, 0, 0, (uint32_t)i, 3);
    const double um = unit53(u.x, u.y), umu = unit53(u.z, u.w);
    const Q4d dq = qexp_d(sigma_r * n[3], sigma_r * n[4], sigma_r * n[5]);
    const Q4d qn = qnorm_d(qmul_d(dq, {q0.x, q0.y, q0.z, q0.w}));
    pose[2 * i] = make_float4((float)(x0.x + sigma_p * n[0]), (float)(x0.y + sigma_p * n[1]),
                              (float)(x0.z + sigma_p * n[2]), 0.0f);
    pose[2 * i + 1] = make_float4((float)qn.w, (float)qn.x, (float)qn.y, (float)qn.z);
    vel[2 * i] = make_float4(0, 0, 0, 0);
    vel[2 * i + 1] = make_float4(0, 0, 0, 0);
    params[i] = make_float2((float)(m_lo + (m_hi - m_lo) * um), (float)(mu_lo + (mu_hi - mu_lo) * umu));
    status[i] = 0;
}

__device__ __forceinline__ bool fin4(float4 v) {
    return isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w);
}

__global__ void set_state_kernel(int N, int n_shapes, const float4 *pose_in, const float4 *vel_in,
                                 const float2 *params_in, const int *shape_in, const int *iters_in,
                                 float4 *pose, float4 *vel, float2 *params, int *shape, int *iters,
                                 int *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float4 p0 = pose_in[2 * i], p1 = pose_in[2 * i + 1];
    const float4 v0 = vel_in[2 * i], v1 = vel_in[2 * i + 1];
    const float2 th = params_in[i];
    const int sh = shape_in ? shape_in[i] : shape[i];
    const int it = iters_in ? iters_in[i] : iters[i];
    bool ok = fin4(p0) && fin4(p1) && fin4(v0) && fin4(v1) && isfinite(th.x) && isfinite(th.y);
    ok = ok && th.x > 0.0f && th.y >= 0.0f && sh >= 0 && sh < n_shapes && it >= 0 && it <= 4096;
    const float qn = p1.x * p1.x + p1.y * p1.y + p1.z * p1.z + p1.w * p1.w;
    ok = ok && qn > 0.5f && qn < 2.0f;
    pose[2 * i] = make_float4(p0.x, p0.y, p0.z, 0.0f);
    pose[2 * i + 1] = p1;
    vel[2 * i] = make_float4(v0.x, v0.y, v0.z, 0.0f);
    vel[2 * i + 1] = make_float4(v1.x, v1.y, v1.z, 0.0f);
    params[i] = th;
    shape[i] = (sh >= 0 && sh < n_shapes) ? sh : 0;
    iters[i] = (it >= 0 && it <= 4096) ? it : 0;
    status[i] = ok ? 0 : IH_ENV_INVALID;
}

// Work order of the environments, most expensive first (longest processing
// time first), by a counting sort on a bucketed estimate S * iters.
constexpr int kLptBuckets = 64;

__device__ __forceinline__ int lpt_bucket(const int *shape_count, const int *shape, const int *iters, int i) {
    const float cost = (float)shape_count[shape[i]] * (float)max(iters[i], 1);
    const int b = (int)(log2f(cost) * 3.0f);
    return kLptBuckets - 1 - min(max(b, 0), kLptBuckets - 1);
}

__global__ void lpt_hist_kernel(int N, const int *shape_count, const int *shape, const int *iters, int *hist) {
    __shared__ int h[kLptBuckets];
    if (threadIdx.x < kLptBuckets) h[threadIdx.x] = 0;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        atomicAdd(&h[lpt_bucket(shape_count, shape, iters, i)], 1);
    __syncthreads();
    if (threadIdx.x < kLptBuckets && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void lpt_scan_kernel(int *hist) {
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < kLptBuckets; ++b) { const int c = hist[b]; hist[b] = acc; acc += c; }
    }
}

// One warp walks the environments in index order, 32 at a time, so that the
// order within a bucket is the index order (a stable sort).
__global__ void lpt_scatter_kernel(int N, const int *shape_count, const int *shape, const int *iters, const int *offs,
                                   int *order) {
    __shared__ int next[kLptBuckets];
    const int lane = threadIdx.x;
    for (int b = lane; b < kLptBuckets; b += 32) next[b] = offs[b];
    __syncwarp();
    for (int base = 0; base < N; base += 32) {
        const int i = base + lane;
        const int b = i < N ? lpt_bucket(shape_count, shape, iters, i) : kLptBuckets;   // sentinel
        const unsigned same = __match_any_sync(0xffffffffu, b);
        const int rank = __popc(same & ((1u << lane) - 1u));
        const int leader = __ffs(same) - 1;
        int start = 0;
        if (i < N) start = next[b];
        __syncwarp();
        if (i < N) order[start + rank] = i;
        if (i < N && lane == leader) next[b] = start + __popc(same);
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_lpt_order(int N, const int *shape_count, const int *shape, const int *iters, int *scratch,
                             int *order, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(scratch, 0, kLptBuckets * sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int blocks = min(152 * 4, (N + 255) / 256);
    lpt_hist_kernel<<<blocks, 256, 0, s>>>(N, shape_count, shape, iters, scratch);
    lpt_scan_kernel<<<1, 32, 0, s>>>(scratch);
    lpt_scatter_kernel<<<1, 32, 0, s>>>(N, shape_count, shape, iters, scratch, order);
    return cudaGetLastError();
}

cudaError_t launch_shape_setup(const float4 *spheres_in, float4 *spheres_out, const int *first,
                               const int *count, int n_shapes, float *jinv, float *bound,
                               const int *cl_first, float4 *clusters, cudaStream_t s) {
    shape_setup_kernel<<<n_shapes, 256, 0, s>>>(spheres_in, spheres_out, first, count, jinv, bound, cl_first,
                                                clusters);
    return cudaGetLastError();
}

cudaError_t launch_fk(const DevScene &sc, const float *q, int n_frames, int substeps,
                      float4 *link_tab_out, cudaStream_t s) {
    const int per = sc.n_fingers > 0 ? sc.n_fingers : 1;
    const int n = n_frames * (substeps + 1) * per;
    fk_kernel<<<(n + 127) / 128, 128, 0, s>>>(sc, q, n_frames, substeps, link_tab_out);
    return cudaGetLastError();
}

cudaError_t launch_sample_initial(int N, float4 pose0, float4 quat0, float sigma_p, float sigma_r,
                                  float m_lo, float m_hi, float mu_lo, float mu_hi, uint64_t seed,
                                  float4 *pose, float4 *vel, float2 *params, int *status,
                                  cudaStream_t s) {
    sample_initial_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, pose0, quat0, sigma_p, sigma_r, m_lo, m_hi,
                                                          mu_lo, mu_hi, seed, pose, vel, params, status);
    return cudaGetLastError();
}

cudaError_t launch_set_state(int N, int n_shapes, const float *pose, const float *vel,
                             const float *params, const int *shape_in, const int *iters_in,
                             float4 *pose_out, float4 *vel_out, float2 *params_out, int *shape,
                             int *iters, int *status, cudaStream_t s) {
    set_state_kernel<<<(N + 127) / 128, 128, 0, s>>>(
        N, n_shapes, reinterpret_cast<const float4 *>(pose), reinterpret_cast<const float4 *>(vel),
        reinterpret_cast<const float2 *>(params), shape_in, iters_in, pose_out, vel_out, params_out,
        shape, iters, status);
    return cudaGetLastError();
}

}  // namespace ih
