// optim.cu -- the periodic optimizer update (Sec. III-D, population-based
// variant with elite-weighted Gaussian exploration; Algorithm 1, "update
// simulations according to optimizer").
//
// select (one CTA of 1024 threads, FP64 statistics):
//   window means C_i -> 64-bit order-preserving keys (NaN = +inf); radix
//   select of the k-th smallest key in eight 8-bit passes; elites = keys below
//   it plus the lowest-index ties; i* = smallest (key, index); elite weights
//   exp(-(C - C_min)/s); their CDF in index order; weighted mean and
//   covariance of z = [x, log(R R_{i*}^T), m, mu]; 8x8 Cholesky of
//   Sigma_w + Sigma_floor; the resampling offset u.
// apply (one thread per environment):
//   non-elite i with rank r takes the elite at CDF position (u + r)/(N - k),
//   copies its state and adds L eps (Philox normals); every window sum resets.
#include "internal.cuh"

namespace ih {
namespace {

constexpr int kSel = 1024;
constexpr int kWarps = kSel / 32;

__device__ __forceinline__ unsigned long long order_key(double c) {
    if (isnan(c)) c = INFINITY;
    const unsigned long long b = (unsigned long long)__double_as_longlong(c);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum of `n` doubles per thread (n <= 36); result valid in thread 0's out
template <int NV>
__device__ void block_sum(double (&v)[NV], double (*red)[NV], double (&out)[NV]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0)
        for (int k = 0; k < NV; ++k) red[wid][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < kWarps; ++w) s += red[w][k];
            out[k] = s;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ double mean_of(const double *c_sum, int i, double n) {
    return __ddiv_rn(c_sum[i], n);
}

__global__ void __launch_bounds__(kSel) select_kernel(const OptArgs a) {
    __shared__ unsigned int hist[256];
    __shared__ unsigned long long s_prefix;
    __shared__ unsigned int s_rem;
    __shared__ unsigned int s_scan[kSel];
    __shared__ double red8[kWarps][8];
    __shared__ double red36[kWarps][36];
    __shared__ double s8[8];
    __shared__ double s36[36];
    __shared__ double s_misc[4];
    __shared__ unsigned long long s_min_key;
    __shared__ int s_min_idx;

    const int N = a.N, t = threadIdx.x;
    const double n = (double)(*a.n_window);
    int k = (int)floor((double)a.elite_frac * (double)N);
    if (k < 1) k = 1;
    if (k > N) k = N;
    const int chunk = (N + kSel - 1) / kSel;
    const int lo = t * chunk, hi = min(N, lo + chunk);

    // ---- radix select of the k-th smallest key
    if (t == 0) { s_prefix = 0ull; s_rem = (unsigned)k; }
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        if (t < 256) hist[t] = 0u;
        __syncthreads();
        const unsigned long long pre = s_prefix;
        const unsigned long long hmask = (pass == 0) ? 0ull : (~0ull << (shift + 8));
        for (int i = t; i < N; i += kSel) {
            const unsigned long long key = order_key(mean_of(a.c_sum, i, n));
            if ((key & hmask) == pre) atomicAdd(&hist[(key >> shift) & 0xff], 1u);
        }
        __syncthreads();
        if (t == 0) {
            unsigned rem = s_rem, acc = 0;
            int b = 0;
            for (; b < 256; ++b) {
                if (acc + hist[b] >= rem) break;
                acc += hist[b];
            }
            s_rem = rem - acc;
            s_prefix = pre | ((unsigned long long)b << shift);
        }
        __syncthreads();
    }
    const unsigned long long T = s_prefix;
    const unsigned need_eq = s_rem;   // elites taken from the keys equal to T, lowest index first

    // ---- elite flags in index order: ties broken by a scan over equal keys
    unsigned eq_local = 0;
    for (int i = lo; i < hi; ++i) eq_local += (order_key(mean_of(a.c_sum, i, n)) == T);
    s_scan[t] = eq_local;
    __syncthreads();
    for (int o = 1; o < kSel; o <<= 1) {   // inclusive Hillis-Steele scan
        const unsigned v = (t >= o) ? s_scan[t - o] : 0u;
        __syncthreads();
        s_scan[t] += v;
        __syncthreads();
    }
    unsigned eq_before = s_scan[t] - eq_local;
    __syncthreads();
    unsigned el_local = 0;
    for (int i = lo; i < hi; ++i) {
        const unsigned long long key = order_key(mean_of(a.c_sum, i, n));
        bool e = key < T;
        if (key == T) { e = eq_before < need_eq; ++eq_before; }
        a.is_elite[i] = e;
        el_local += e;
    }
    s_scan[t] = el_local;
    __syncthreads();
    for (int o = 1; o < kSel; o <<= 1) {
        const unsigned v = (t >= o) ? s_scan[t - o] : 0u;
        __syncthreads();
        s_scan[t] += v;
        __syncthreads();
    }
    {
        unsigned er = s_scan[t] - el_local;         // elites before my chunk
        unsigned nr = (unsigned)lo - er;            // non-elites before my chunk
        for (int i = lo; i < hi; ++i) {
            if (a.is_elite[i]) { a.rank[i] = (int)er; a.elite_env[er] = i; ++er; }
            else { a.rank[i] = (int)nr; ++nr; }
        }
    }

    // ---- i* = smallest (key, index)
    unsigned long long bk = ~0ull;
    int bi = 0x7fffffff;
    for (int i = t; i < N; i += kSel) {
        const unsigned long long key = order_key(mean_of(a.c_sum, i, n));
        if (key < bk || (key == bk && i < bi)) { bk = key; bi = i; }
    }
    if (t == 0) { s_min_key = ~0ull; s_min_idx = 0x7fffffff; }
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ok < bk || (ok == bk && oi < bi)) { bk = ok; bi = oi; }
    }
    if ((t & 31) == 0) {
        // serialise the 32 warp winners through one lock-free min on the packed pair
        atomicMin(&s_min_key, bk);
    }
    __syncthreads();
    if ((t & 31) == 0 && bk == s_min_key) atomicMin(&s_min_idx, bi);
    __syncthreads();
    const int istar = s_min_idx;
    const double cmin_raw = mean_of(a.c_sum, istar, n);
    const double cmin = isnan(cmin_raw) ? INFINITY : cmin_raw;

    // ---- elite weights: exp(-(C - C_min)/s), s = population std of finite elite costs
    double acc2[2] = {0.0, 0.0};   // sum, count of finite elite costs
    for (int j = t; j < k; j += kSel) {
        const double c = mean_of(a.c_sum, a.elite_env[j], n);
        if (isfinite(c)) { acc2[0] += c; acc2[1] += 1.0; }
    }
    {
        double out2[2];
        block_sum<2>(acc2, reinterpret_cast<double(*)[2]>(red8), out2);
        if (t == 0) { s_misc[0] = out2[0]; s_misc[1] = out2[1]; }
        __syncthreads();
    }
    const double nfin = s_misc[1];
    const double cmean = nfin > 0 ? s_misc[0] / nfin : 0.0;
    double accv[1] = {0.0};
    for (int j = t; j < k; j += kSel) {
        const double c = mean_of(a.c_sum, a.elite_env[j], n);
        if (isfinite(c)) accv[0] += (c - cmean) * (c - cmean);
    }
    {
        double out1[1];
        block_sum<1>(accv, reinterpret_cast<double(*)[1]>(red8), out1);
        if (t == 0) s_misc[2] = nfin > 0 ? sqrt(out1[0] / nfin) : 0.0;
        __syncthreads();
    }
    const double sd = s_misc[2];
    // unnormalised weights into elite_cdf, then their sum
    double accw[1] = {0.0};
    for (int j = t; j < k; j += kSel) {
        const double c = mean_of(a.c_sum, a.elite_env[j], n);
        double w;
        if (nfin == 0.0) w = 1.0;
        else if (!isfinite(c)) w = 0.0;
        else if (!(sd >= 1e-12)) w = 1.0;
        else w = exp(-(c - cmin) / sd);
        a.elite_cdf[j] = w;
        accw[0] += w;
    }
    {
        double out1[1];
        block_sum<1>(accw, reinterpret_cast<double(*)[1]>(red8), out1);
        if (t == 0) s_misc[3] = out1[0];
        __syncthreads();
    }
    const double wsum = s_misc[3];

    // ---- weighted mean and covariance of z over the elites with w > 0
    const float4 qr4 = a.pose[2 * istar + 1];
    const Q4d qref_conj = {qr4.x, -qr4.y, -qr4.z, -qr4.w};
    double zs[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = t; j < k; j += kSel) {
        const double w = a.elite_cdf[j] / wsum;
        if (w == 0.0) continue;
        const int e = a.elite_env[j];
        const float4 p0 = a.pose[2 * e], p1 = a.pose[2 * e + 1];
        double lr[3];
        qlog_d(qmul_d({p1.x, p1.y, p1.z, p1.w}, qref_conj), lr);
        const float2 th = a.params[e];
        const double z[8] = {p0.x, p0.y, p0.z, lr[0], lr[1], lr[2], th.x, th.y};
        for (int c = 0; c < 8; ++c) zs[c] += w * z[c];
    }
    block_sum<8>(zs, red8, s8);
    double cs[36];
    for (int c = 0; c < 36; ++c) cs[c] = 0.0;
    for (int j = t; j < k; j += kSel) {
        const double w = a.elite_cdf[j] / wsum;
        if (w == 0.0) continue;
        const int e = a.elite_env[j];
        const float4 p0 = a.pose[2 * e], p1 = a.pose[2 * e + 1];
        double lr[3];
        qlog_d(qmul_d({p1.x, p1.y, p1.z, p1.w}, qref_conj), lr);
        const float2 th = a.params[e];
        const double z[8] = {p0.x, p0.y, p0.z, lr[0], lr[1], lr[2], th.x, th.y};
        double d[8];
        for (int c = 0; c < 8; ++c) d[c] = z[c] - s8[c];
        int q = 0;
        for (int r = 0; r < 8; ++r)
            for (int c = 0; c <= r; ++c) cs[q++] += w * d[r] * d[c];
    }
    block_sum<36>(cs, red36, s36);

    // ---- normalised weights -> inclusive CDF in elite index order (serial, FP64)
    if (t == 0) {
        double cum = 0.0;
        for (int j = 0; j < k; ++j) {
            cum += a.elite_cdf[j] / wsum;
            a.elite_cdf[j] = cum;
        }
        // Cholesky of Sigma_w + diag(floor^2), lower triangle, row-major 8x8
        double A[8][8], L[8][8];
        int q = 0;
        for (int r = 0; r < 8; ++r)
            for (int c = 0; c <= r; ++c) { A[r][c] = s36[q]; A[c][r] = s36[q]; ++q; }
        for (int r = 0; r < 8; ++r) A[r][r] += a.floor_var[r];
        bool ok = true;
        for (int r = 0; r < 8; ++r)
            for (int c = 0; c < 8; ++c) L[r][c] = 0.0;
        for (int i = 0; i < 8 && ok; ++i)
            for (int j = 0; j <= i; ++j) {
                double s = A[i][j];
                for (int m = 0; m < j; ++m) s -= L[i][m] * L[j][m];
                if (i == j) {
                    if (!(s > 0.0)) { ok = false; break; }
                    L[i][i] = sqrt(s);
                } else {
                    L[i][j] = s / L[j][j];
                }
            }
        for (int r = 0; r < 8; ++r)
            for (int c = 0; c < 8; ++c) a.chol[8 * r + c] = L[r][c];
        const uint4 uw = rng_words(a.seed, 2, a.update_index, 0, 0);
        a.chol[64] = (double)k;
        a.chol[65] = unit53(uw.x, uw.y);
        a.chol[66] = (double)istar;
        a.chol[67] = ok ? 1.0 : 0.0;
        *a.argmin_state = istar;
        if (a.argmin_out) *a.argmin_out = istar;
    }
}

__global__ void apply_kernel(const OptArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = a.N;
    if (i >= N) return;
    if (i == 0) *a.n_window_reset = 0;
    a.c_sum_reset[i] = 0.0;
    if (a.is_elite[i]) {
        if (a.parent_out) a.parent_out[i] = i;
        return;
    }
    const int k = (int)a.chol[64];
    const double u = a.chol[65];
    const bool ok = a.chol[67] != 0.0;
    const int M = N - k;
    const double pos = __ddiv_rn(u + (double)a.rank[i], (double)M);
    // first elite whose inclusive CDF exceeds pos (the last one if rounding left none)
    int lo = 0, hi = k - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (pos < a.elite_cdf[mid]) hi = mid; else lo = mid + 1;
    }
    const int par = a.elite_env[lo];
    if (a.parent_out) a.parent_out[i] = par;
    if (!ok) return;
    double eps[8], d[8];
    for (int b = 0; b < 4; ++b) gauss2(rng_words(a.seed, 1, a.update_index, (uint32_t)i, (uint32_t)b), eps[2 * b], eps[2 * b + 1]);
    for (int r = 0; r < 8; ++r) {
        double s = 0.0;
        for (int c = 0; c <= r; ++c) s += a.chol[8 * r + c] * eps[c];
        d[r] = s;
    }
    const float4 p0 = a.pose[2 * par], p1 = a.pose[2 * par + 1];
    const Q4d qn = qnorm_d(qmul_d(qexp_d(d[3], d[4], d[5]), {p1.x, p1.y, p1.z, p1.w}));
    a.pose[2 * i] = make_float4((float)(p0.x + d[0]), (float)(p0.y + d[1]), (float)(p0.z + d[2]), 0.0f);
    a.pose[2 * i + 1] = make_float4((float)qn.w, (float)qn.x, (float)qn.y, (float)qn.z);
    a.vel[2 * i] = a.vel[2 * par];
    a.vel[2 * i + 1] = a.vel[2 * par + 1];
    const float2 th = a.params[par];
    const double m = fmin(fmax((double)th.x + d[6], (double)a.m_lo), (double)a.m_hi);
    const double mu = fmin(fmax((double)th.y + d[7], (double)a.mu_lo), (double)a.mu_hi);
    a.params[i] = make_float2((float)m, (float)mu);
    a.status[i] = a.status[par];
}

}  // namespace

cudaError_t launch_optimizer(const OptArgs &a, cudaStream_t s) {
    select_kernel<<<1, kSel, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    apply_kernel<<<(a.N + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ih
