// optim.cu -- the periodic optimizer update (Sec. III-D, population-based
// variant with elite-weighted Gaussian exploration; Algorithm 1, "update
// simulations according to optimizer").
//
// FP64 issue is scarce on this part, so the update is split so that every
// FP64 transcendental runs in a grid spread over the SMs:
//   select    (1 CTA)  order-preserving 64-bit keys of the window means
//                      (NaN = +inf); radix select of the k-th smallest key in
//                      eight 8-bit passes; elite flags (lowest index first
//                      among equal keys), ranks, i*, mean and standard
//                      deviation of the finite elite costs; resampling offset.
//   stats     (grid)   per elite: w = exp(-(C - C_min)/s); z - z_{i*} with
//                      z = [x, log(R R_{i*}^T), m, mu]; per-block weighted
//                      moments and the inclusive prefix of w within the block.
//   finalize  (1 CTA)  sums the moments, weighted mean and covariance,
//                      L = chol(Sigma_w + Sigma_floor), block offsets of w.
//   apply     (grid)   non-elite i of rank r takes the elite whose cumulative
//                      weight first exceeds (u + r)/(N - k) of the total, copies
//                      its state, adds L eps (Philox normals), clamps m and mu;
//                      every window sum restarts.
#include <cmath>

#include "internal.cuh"

namespace ih {
namespace {

constexpr int kSel = 1024;            // threads of the select kernel for large N
constexpr int kSelSmall = 256;        // ... for N <= kKeys * kSelSmall
constexpr int kKeys = 8;              // keys per thread held in registers
constexpr int kFin = 128;             // threads of the finalize kernel

enum { M_K = 64, M_U, M_ISTAR, M_OK, M_WSUM, M_CMIN, M_SD, M_NFIN, M_NBLK };

// Programmatic dependent launch: the kernels of the update are launched so
// that each may be scheduled while the one before it drains; each waits here,
// before its first read of that kernel's results, until it has completed and
// its writes are visible (at once when launched without the dependency).
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... P, typename... A>
cudaError_t launch_dependent(void (*k)(P...), int grid, int block, cudaStream_t s, A... args) {
    cudaLaunchConfig_t c = {};
    c.gridDim = dim3(grid);
    c.blockDim = dim3(block);
    c.dynamicSmemBytes = 0;
    c.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    c.attrs = at;
    c.numAttrs = 1;
    return cudaLaunchKernelEx(&c, k, args...);
}

// NaN and finiteness tests on the bits (integer instructions: FP64 compares
// take the scarce FP64 pipe)
__device__ __forceinline__ bool nan_bits(double c) {
    return ((unsigned long long)__double_as_longlong(c) & 0x7fffffffffffffffull) > 0x7ff0000000000000ull;
}
__device__ __forceinline__ bool finite_bits(double c) {
    return ((unsigned long long)__double_as_longlong(c) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

__device__ __forceinline__ unsigned long long order_key(double c) {
    const unsigned long long b =
        nan_bits(c) ? 0x7ff0000000000000ull : (unsigned long long)__double_as_longlong(c);   // NaN = +inf
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide inclusive scan of one unsigned per thread: warp scans, then a
// scan of the warp totals by the first warp (buf holds NT / 32 + 1 entries)
template <int NT>
__device__ unsigned block_scan(unsigned v, unsigned *buf) {
    constexpr int kWarps = NT / 32;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) buf[w] = v;
    __syncthreads();
    if (w == 0) {
        unsigned x = lane < kWarps ? buf[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane < kWarps) buf[lane] = x;
    }
    __syncthreads();
    const unsigned r = v + (w > 0 ? buf[w - 1] : 0u);
    __syncthreads();
    return r;
}

// block sum of one double per thread, where only the first nw warps can hold
// nonzero values (the others issue no FP64 work): warp sums, then the warps'
// partials in warp order by thread 0 (the omitted partials are zeros)
template <int NT>
__device__ double block_sum(double v, double *red, int nw = NT / 32) {
    if ((int)(threadIdx.x >> 5) < nw) {
        v = warp_sum(v);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    }
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; ++w) s += red[w];
    __syncthreads();
    return s;   // valid in thread 0
}

template <int NT>
__global__ void __launch_bounds__(NT) select_kernel(const OptArgs a) {
    constexpr int kSel = NT, kWarps = NT / 32;
    // the small instance (N <= kKeys kSelSmall) stages the window means and
    // the elite list in shared memory; the large one reads them from global
    // memory (read-only here: c_mean through the non-coherent path)
    constexpr bool kStage = NT == kSelSmall;
    __shared__ double s_cost[kStage ? kKeys * kSelSmall : 1];
    __shared__ int s_elite[kStage ? kKeys * kSelSmall : 1];
    __shared__ unsigned int hist[256];
    __shared__ unsigned long long s_prefix, s_mask;
    __shared__ unsigned int s_rem;
    __shared__ int s_done;
    __shared__ unsigned int s_scan[kWarps + 1];
    __shared__ double red[kWarps];
    __shared__ int s_cnt[kWarps];
    __shared__ double s_val[3];
    __shared__ unsigned long long s_min_key;
    __shared__ int s_min_idx;

    grid_dependency_wait();
    const int N = a.N, t = threadIdx.x;
    int k = (int)floor((double)a.elite_frac * (double)N);
    k = max(1, min(k, N));
    if (t == 0) {   // the elite count and the resampling offset, off the critical path
        const uint32_t upd = a.win ? a.win->update_index : a.update_index;
        const uint4 uw = rng_words(a.seed, 2, upd, 0, 0);
        a.misc[M_K] = (double)k;
        a.misc[M_U] = unit53(uw.x, uw.y);
    }
    const int chunk = (N + kSel - 1) / kSel;
    const int lo = min(N, t * chunk), hi = min(N, lo + chunk);
    auto cost = [&](int i) -> double {
        if constexpr (kStage) return s_cost[i];
        else return __ldg(a.c_mean + i);
    };

    // ---- keys (held in registers when N <= 8 kSel) and i* = smallest (key, index)
    const bool in_regs = N <= kKeys * kSel;
    unsigned long long kreg[kKeys];
    unsigned long long bk = ~0ull;
    int bi = 0x7fffffff;
#pragma unroll
    for (int q = 0; q < kKeys; ++q) {
        const int i = t + q * kSel;
        kreg[q] = 0ull;
        if (in_regs && i < N) {
            const double c = __ldg(a.c_mean + i);
            if constexpr (kStage) s_cost[i] = c;
            kreg[q] = order_key(c);
            if (kreg[q] < bk) { bk = kreg[q]; bi = i; }   // (i ascending: the first of equal keys)
        }
    }
    if (!in_regs) {
        for (int i = t; i < N; i += kSel) {
            const unsigned long long key = order_key(__ldg(a.c_mean + i));
            if (key < bk) { bk = key; bi = i; }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ok < bk || (ok == bk && oi < bi)) { bk = ok; bi = oi; }
    }
    if (t == 0) {
        s_min_key = ~0ull; s_min_idx = 0x7fffffff;
        s_prefix = 0ull; s_mask = 0ull; s_rem = (unsigned)k; s_done = 0;
    }
    __syncthreads();
    if ((t & 31) == 0) atomicMin(&s_min_key, bk);
    __syncthreads();
    if ((t & 31) == 0 && bk == s_min_key) atomicMin(&s_min_idx, bi);

    // ---- radix select of the k-th smallest key
    // The passes stop early once every key whose leading digits equal the
    // prefix found so far is needed: the elites are then exactly the keys whose
    // leading digits are at most the prefix, whatever their remaining digits.
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        if (t < 256) hist[t] = 0u;
        __syncthreads();
        const unsigned long long pre = s_prefix;
        const unsigned long long hmask = (pass == 0) ? 0ull : (~0ull << (shift + 8));
        // histogram of the next digit; lanes of a warp with the same digit add
        // once (leading bytes of similar costs all fall in one bin)
        auto count = [&](bool valid, unsigned long long key) {
            const unsigned bin = valid && (key & hmask) == pre ? (unsigned)((key >> shift) & 0xff) : 0x100u;
            const unsigned same = __match_any_sync(0xffffffffu, bin);
            if (bin < 0x100u && (__ffs(same) - 1) == (t & 31)) atomicAdd(&hist[bin], (unsigned)__popc(same));
        };
        if (in_regs) {
#pragma unroll
            for (int q = 0; q < kKeys; ++q) count(t + q * kSel < N, kreg[q]);
        } else {
            for (int i0 = 0; i0 < N; i0 += kSel) {
                const int i = i0 + t;
                count(i < N, i < N ? order_key(__ldg(a.c_mean + i)) : 0ull);
            }
        }
        __syncthreads();
        if (t < 32) {   // the first bin whose running count reaches rem (warp-parallel scan)
            const unsigned rem = s_rem;
            unsigned c8[8], sum = 0u;
#pragma unroll
            for (int q = 0; q < 8; ++q) { c8[q] = hist[8 * t + q]; sum += c8[q]; }
            unsigned inc = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned u = __shfl_up_sync(0xffffffffu, inc, o);
                if (t >= o) inc += u;
            }
            const unsigned excl = inc - sum;
            // lanes whose range holds the crossing (the last lane holds bin 255 as the fallback)
            const bool here = (excl < rem && inc >= rem) || (t == 31 && inc < rem);
            const unsigned who = __ballot_sync(0xffffffffu, here);
            if (t == __ffs(who) - 1) {
                // the first of the lane's bins whose running count reaches rem (else its last)
                unsigned acc = excl, cb = c8[7];
                int b = 8 * t + 7;
                bool found = false;
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    if (found) continue;
                    if (acc + c8[q] >= rem) { found = true; b = 8 * t + q; cb = c8[q]; }
                    else acc += c8[q];
                }
                s_rem = rem - acc;
                s_prefix = pre | ((unsigned long long)b << shift);
                s_mask = ~0ull << shift;
                if (cb == rem - acc) s_done = 1;
            }
        }
        __syncthreads();
        if (s_done) break;
    }
    const unsigned long long T = s_prefix, M = s_mask;   // M: the digits decided (all 64 after 8 passes)
    const unsigned need_eq = s_rem;   // elites among the keys whose digits under M equal T, lowest index first
    const int istar = s_min_idx;

    // ---- elite flags in index order (the flag of a key equal to T under M
    // depends on the equal keys before it), then ranks: elites and non-elites
    // each numbered in index order
    unsigned eq_local = 0;
    for (int i = lo; i < hi; ++i) eq_local += ((order_key(cost(i)) & M) == T);
    const unsigned eq0 = block_scan<NT>(eq_local, s_scan) - eq_local;
    unsigned el_local = 0;
    {
        unsigned eqb = eq0;
        for (int i = lo; i < hi; ++i) {
            const unsigned long long key = order_key(cost(i)) & M;
            const bool e = key < T || (key == T && eqb++ < need_eq);
            a.is_elite[i] = e;
            el_local += e;
        }
    }
    {
        unsigned er = block_scan<NT>(el_local, s_scan) - el_local;   // elites before my chunk
        unsigned nr = (unsigned)lo - er;                          // non-elites before my chunk
        unsigned eqb = eq0;
        for (int i = lo; i < hi; ++i) {
            const unsigned long long key = order_key(cost(i)) & M;
            if (key < T || (key == T && eqb++ < need_eq)) {
                a.rank[i] = (int)er;
                a.elite_env[er] = i;
                if constexpr (kStage) s_elite[er] = i;
                ++er;
            } else {
                a.rank[i] = (int)nr;
                ++nr;
            }
        }
    }
    __syncthreads();   // the elite list (global and staged) is complete
    auto elite = [&](int j) -> int {
        if constexpr (kStage) return s_elite[j];
        else return a.elite_env[j];
    };

    // ---- mean and population standard deviation of the finite elite costs
    // (the warps past the elites hold zeros and skip the sums)
    const int nw = min(kWarps, (k + 31) / 32);
    double sum = 0.0;
    int cnt = 0;
    for (int j = t; j < k; j += kSel) {
        const double c = cost(elite(j));
        if (finite_bits(c)) { sum += c; ++cnt; }
    }
    const double tot = block_sum<NT>(sum, red, nw);
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if ((t & 31) == 0) s_cnt[t >> 5] = cnt;
    __syncthreads();
    if (t == 0) {
        int nf = 0;
        for (int w = 0; w < kWarps; ++w) nf += s_cnt[w];
        s_val[0] = tot; s_val[1] = (double)nf;
        s_val[2] = nf > 0 ? tot / (double)nf : 0.0;   // the mean, divided once
    }
    __syncthreads();
    const double mean = s_val[2];
    double sq = 0.0;
    for (int j = t; j < k; j += kSel) {
        const double c = cost(elite(j));
        if (finite_bits(c)) sq += (c - mean) * (c - mean);
    }
    const double ss = block_sum<NT>(sq, red, nw);
    if (t == 0) {
        const double nf = s_val[1];
        const double c0 = cost(istar);
        a.misc[M_ISTAR] = (double)istar;
        a.misc[M_CMIN] = nan_bits(c0) ? INFINITY : c0;
        a.misc[M_SD] = nf > 0 ? sqrt(ss / nf) : 0.0;
        a.misc[M_NFIN] = nf;
        *a.argmin_state = istar;
        if (a.argmin_out) *a.argmin_out = istar;
    }
}

// One elite per lane (index order), kOptBlock elites per block, four warps:
// the weight and its in-block prefix (warp 0), the rotation offset through the
// FP64 log map (warp 1) and the other offsets (warp 2) are formed side by
// side, then each warp forms a quarter of the 45 moment products. FP64
// instructions are scarce on this part; split so, each warp issues few.
constexpr int kStatWarps = 4;
// the factors of moment q: (a << 4) | b, with w = w e_0 e_0, w d_r = w e_{1+r}
// e_0 and w d_r d_c = w e_{1+r} e_{1+c} (c <= r) in the order of kMoments
__constant__ unsigned char c_mom_ab[kMoments] = {
    0x00, 0x10, 0x20, 0x30, 0x40, 0x50, 0x60, 0x70, 0x80,
    0x11,
    0x21, 0x22,
    0x31, 0x32, 0x33,
    0x41, 0x42, 0x43, 0x44,
    0x51, 0x52, 0x53, 0x54, 0x55,
    0x61, 0x62, 0x63, 0x64, 0x65, 0x66,
    0x71, 0x72, 0x73, 0x74, 0x75, 0x76, 0x77,
    0x81, 0x82, 0x83, 0x84, 0x85, 0x86, 0x87, 0x88};
__global__ void __launch_bounds__(kOptBlock * kStatWarps) stats_kernel(const OptArgs a) {
    __shared__ double s_w[kOptBlock];
    __shared__ double s_d[kOptBlock][9];   // (1, offsets): moment q = w e_{a(q)} e_{b(q)}
    __shared__ double tm[kOptBlock][kMoments + 1];
    grid_dependency_wait();
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int j = blockIdx.x * kOptBlock + lane;
    const int k = (int)a.misc[M_K];
    const int istar = (int)a.misc[M_ISTAR];
    const bool valid = j < k;
    const int e = valid ? a.elite_env[j] : 0;
    if (wq == 0) {   // w = exp(-(C - C_min)/s)
        const double cmin = a.misc[M_CMIN], sd = a.misc[M_SD], nfin = a.misc[M_NFIN];
        double w = 0.0;
        if (valid) {
            const double c = a.c_mean[e];
            if (nfin == 0.0) w = 1.0;
            else if (!finite_bits(c)) w = 0.0;
            else if (!(sd >= 1e-12)) w = 1.0;
            else w = exp(-(c - cmin) / sd);
        }
        s_w[lane] = w;
        // inclusive prefix of w within the block (index order), and the block total
        double pre = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double v = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += v;
        }
        if (valid) a.elite_w[j] = pre;
        if (lane == 31) a.block_w[blockIdx.x] = pre;
    } else if (wq == 1) {   // log(R R_{i*}^T): the offset of the rotation coordinate (0 at i*)
        double lr[3] = {0.0, 0.0, 0.0};
        if (valid) {
            const float4 p1 = a.pose[2 * e + 1], r1 = a.pose[2 * istar + 1];
            qlog_d(qmul_d({p1.x, p1.y, p1.z, p1.w}, {r1.x, -r1.y, -r1.z, -r1.w}), lr);
        }
        s_d[lane][4] = lr[0]; s_d[lane][5] = lr[1]; s_d[lane][6] = lr[2];
    } else if (wq == 2) {   // position, mass and friction offsets from z_{i*}
        double d0 = 0.0, d1 = 0.0, d2 = 0.0, d6 = 0.0, d7 = 0.0;
        if (valid) {
            const float4 p0 = a.pose[2 * e], r0 = a.pose[2 * istar];
            const float2 th = a.params[e], tr = a.params[istar];
            d0 = (double)p0.x - r0.x; d1 = (double)p0.y - r0.y; d2 = (double)p0.z - r0.z;
            d6 = (double)th.x - tr.x; d7 = (double)th.y - tr.y;
        }
        s_d[lane][0] = 1.0;
        s_d[lane][1] = d0; s_d[lane][2] = d1; s_d[lane][3] = d2; s_d[lane][7] = d6; s_d[lane][8] = d7;
    }
    __syncthreads();
    // moments (w, w d, w d d^T lower triangle; zero for an elite of weight 0):
    // moment q = (w e_a) e_b with e = (1, d), warp wq forming q = wq, wq + 4, ...
    // (the same code on every warp: no divergent branches to serialise)
    {
        const double w = s_w[lane];
        const bool pos = valid && w > 0.0;
#pragma unroll
        for (int m = 0; m < (kMoments + kStatWarps - 1) / kStatWarps; ++m) {
            const int q = wq + kStatWarps * m;
            if (q < kMoments) {
                const int ab = c_mom_ab[q];
                const double v = w * s_d[lane][ab >> 4] * s_d[lane][ab & 15];
                tm[lane][q] = pos ? v : 0.0;
            }
        }
    }
    __syncthreads();
    // block sums of the moments: moment q summed over the block's elites in
    // index order by thread q
    if (threadIdx.x < kMoments) {
        double sacc = 0.0;
        for (int r = 0; r < kOptBlock; ++r) sacc += tm[r][threadIdx.x];
        a.moments[(size_t)blockIdx.x * kMoments + threadIdx.x] = sacc;
    }
}

__global__ void __launch_bounds__(kFin) finalize_kernel(const OptArgs a, int nblocks) {
    constexpr int kSel = kFin, kWarps = kFin / 32;
    __shared__ double sm[kMoments];
    __shared__ double cv[8][8];
    __shared__ double wtot[32];
    __shared__ double s_carry;
    __shared__ double nm[kMoments];
    grid_dependency_wait();
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    // up to 32 blocks the first warp scans their weight sums alone (loaded
    // here, beside the moments)
    const bool one_warp = nblocks <= 32;
    const double vw = (one_warp && t < nblocks) ? a.block_w[t] : 0.0;
    // moments: thread q < 45 sums its moment over the blocks in block order
    if (t < kMoments) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += a.moments[(size_t)b * kMoments + t];
        sm[t] = s;
    }
    // exclusive offsets of the per-block weight sums, in chunks of kSel blocks:
    // warp scans, then the warp totals in warp order by the first warp
    if (t == 0) s_carry = 0.0;
    __syncthreads();
    if (one_warp && wid == 0) {
        double inc = vw;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (t < nblocks) a.block_w[t] = inc - vw;
        const double total = __shfl_sync(0xffffffffu, inc, 31);
        if (lane == 0) s_carry = total;
    }
    for (int base = 0; base < nblocks && !one_warp; base += kSel) {
        const int b = base + t;
        const double v = (b < nblocks) ? a.block_w[b] : 0.0;
        double inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) wtot[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            double x = lane < kWarps ? wtot[lane] : 0.0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double u = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += u;
            }
            if (lane < kWarps) wtot[lane] = x;
        }
        __syncthreads();
        const double carry = s_carry;
        const double before = (wid > 0 ? wtot[wid - 1] : 0.0) + (inc - v);
        if (b < nblocks) a.block_w[b] = carry + before;
        __syncthreads();
        if (t == 0) s_carry = carry + wtot[kWarps - 1];
        __syncthreads();
    }
    // weighted covariance (36 entries in parallel) plus the floor, from the
    // moments divided by the weight sum once each
    const double wsum = sm[0];
    if (t >= 1 && t < kMoments) nm[t] = sm[t] / wsum;
    __syncthreads();
    if (t < 64) {
        const int r = t >> 3, c = t & 7;
        const int hi = r > c ? r : c, lo = r > c ? c : r;
        const double mr = nm[1 + r], mc = nm[1 + c];
        double v = nm[9 + hi * (hi + 1) / 2 + lo] - mr * mc;
        if (r == c) v += a.floor_var[r];
        cv[r][c] = v;
    }
    __syncthreads();
    // Cholesky by the first warp: lane i < 8 holds row i of L; column j in
    // turn, s = C_ij - sum_{m<j} L_im L_jm in m order, L_jj = sqrt(s_jj),
    // L_ij = s_ij / L_jj, both through one reciprocal square root r = 1/L_jj
    // (L_jj = s_jj r, L_ij = s_ij r: the column's chain of scarce FP64
    // instructions is then one rsqrt long instead of a sqrt and a division)
    if (wid == 0) {
        double L[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) L[c] = 0.0;
        bool ok = wsum > 0.0;
        const int i = lane;
        const bool row = i < 8;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            double sj = (row && i >= j) ? cv[i][j] : 0.0;
#pragma unroll
            for (int m = 0; m < j; ++m) {
                const double ljm = __shfl_sync(0xffffffffu, L[m], j);
                if (row && i >= j) sj -= L[m] * ljm;
            }
            const double djj = __shfl_sync(0xffffffffu, sj, j);
            if (!(djj > 0.0)) ok = false;
            const double rj = ok ? rsqrt(djj) : 0.0;
            if (row && i == j) L[j] = djj * rj;
            else if (row && i > j) L[j] = sj * rj;
        }
        if (!ok) {
#pragma unroll
            for (int c = 0; c < 8; ++c) L[c] = 0.0;
        }
        if (i < 8)
            for (int c = 0; c < 8; ++c) a.misc[8 * i + c] = L[c];
        if (lane == 0) {
            a.misc[M_OK] = ok ? 1.0 : 0.0;
            a.misc[M_WSUM] = s_carry;
            a.misc[M_NBLK] = (double)nblocks;
        }
    }
}

__device__ __forceinline__ double cum_w(const OptArgs &a, int j) {
    return a.block_w[j / kOptBlock] + a.elite_w[j];
}

constexpr int kCdfSmem = 2048;   // elites whose CDF apply_kernel stages in shared memory

// Four lanes per environment (a quad): each draws one Box-Muller pair and two
// rows of L eps, so every warp's FP64 chain is a quarter as long; the quad's
// first lane does the resampling search and writes the state.
constexpr int kApplyLanes = 4;

__global__ void __launch_bounds__(kOptBlock * kApplyLanes) apply_kernel(const OptArgs a) {
    __shared__ double cdf[kCdfSmem];
    grid_dependency_wait();
    const int sub = threadIdx.x & (kApplyLanes - 1);
    const int i = blockIdx.x * kOptBlock + (int)(threadIdx.x / kApplyLanes);
    const unsigned qmask = 0xfu << (threadIdx.x & 28u);   // this quad's lanes
    const int N = a.N;
    const int k = (int)a.misc[M_K];
    const bool staged = k <= kCdfSmem;
    if (staged) {   // the block's binary searches read the CDF from shared memory
        for (int j = threadIdx.x; j < k; j += blockDim.x) cdf[j] = cum_w(a, j);
        __syncthreads();
    }
    if (i >= N) return;   // whole quads
    if (sub == 0) {
        if (i == 0) *a.n_window = 0;
        a.c_sum[i] = 0.0;
    }
    if (a.is_elite[i]) {
        if (sub == 0 && a.parent_out) a.parent_out[i] = i;
        return;
    }
    if (sub == 0 && a.cache_n) a.cache_n[i] = 0;   // replaced: its solver starts cold
    const bool ok = a.misc[M_OK] != 0.0;
    int par = 0;
    // the parent's state, requested as soon as the parent is known (elites
    // are never written here)
    float4 pp0, pp1, pv0, pv1;
    float2 pth;
    int pst;
    if (sub == 0) {
        const double u = a.misc[M_U], wsum = a.misc[M_WSUM];
        const int M = N - k;
        // position (u + r)/M of the normalised CDF, compared on the unnormalised one
        const double pos = __ddiv_rn(u + (double)a.rank[i], (double)M) * wsum;
        int lo = 0, hi = k - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (pos < (staged ? cdf[mid] : cum_w(a, mid))) hi = mid; else lo = mid + 1;
        }
        par = a.elite_env[lo];
        if (a.parent_out) a.parent_out[i] = par;
        pp0 = a.pose[2 * par]; pp1 = a.pose[2 * par + 1];
        pv0 = a.vel[2 * par]; pv1 = a.vel[2 * par + 1];
        pth = a.params[par];
        pst = a.status[par];
    }
    if (!ok) return;
    double e0, e1;
    const uint32_t upd = a.win ? a.win->update_index : a.update_index;
    gauss2(rng_words(a.seed, 1, upd, (uint32_t)i, (uint32_t)sub), e0, e1);
    double eps[8];
#pragma unroll
    for (int b = 0; b < kApplyLanes; ++b) {
        eps[2 * b] = __shfl_sync(qmask, e0, b, kApplyLanes);
        eps[2 * b + 1] = __shfl_sync(qmask, e1, b, kApplyLanes);
    }
    double dr[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {   // rows 2 sub and 2 sub + 1 of L eps
        const int r = 2 * sub + h;
        double sacc = 0.0;
        for (int c = 0; c <= r; ++c) sacc += a.misc[8 * r + c] * eps[c];
        dr[h] = sacc;
    }
    double d[8];
#pragma unroll
    for (int b = 0; b < kApplyLanes; ++b) {
        d[2 * b] = __shfl_sync(qmask, dr[0], b, kApplyLanes);
        d[2 * b + 1] = __shfl_sync(qmask, dr[1], b, kApplyLanes);
    }
    if (sub != 0) return;
    const float4 p0 = pp0, p1 = pp1;
    const Q4d qn = qnorm_d(qmul_d(qexp_d(d[3], d[4], d[5]), {p1.x, p1.y, p1.z, p1.w}));
    a.pose[2 * i] = make_float4((float)(p0.x + d[0]), (float)(p0.y + d[1]), (float)(p0.z + d[2]), 0.0f);
    a.pose[2 * i + 1] = make_float4((float)qn.w, (float)qn.x, (float)qn.y, (float)qn.z);
    a.vel[2 * i] = pv0;
    a.vel[2 * i + 1] = pv1;
    const float2 th = pth;
    const double m = fmin(fmax((double)th.x + d[6], (double)a.m_lo), (double)a.m_hi);
    const double mu = fmin(fmax((double)th.y + d[7], (double)a.mu_lo), (double)a.mu_hi);
    a.params[i] = make_float2((float)m, (float)mu);
    a.status[i] = pst;
    if (a.qj) {   // the parent's hand (elites are not written by this kernel)
        const int D = a.D;
        for (int j = 0; j < D; ++j) {
            a.qj[(size_t)i * D + j] = a.qj[(size_t)par * D + j];
            a.qdj[(size_t)i * D + j] = a.qdj[(size_t)par * D + j];
        }
    }
}

// ---------------------------------------------------------------- WRS / REPS
// (Sec. III-D): a PMF over all simulations, N draws with replacement,
// isotropic exploration of every simulation.
constexpr int kSoft = 1024;

// sums of three doubles over the block (every thread gets them): warp sums,
// then the first warp sums the warps' partials and broadcasts the totals
// through shared memory (FP64 adds are scarce on this part: one warp does them)
__device__ void block_sum3(double &x, double &y, double &z, double (*red)[3]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
        z += __shfl_xor_sync(0xffffffffu, z, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red[wid][0] = x; red[wid][1] = y; red[wid][2] = z; }
    __syncthreads();
    if (wid == 0) {
        double a = red[lane][0], b = red[lane][1], c = red[lane][2];   // kSoft / 32 == 32 partials
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        __syncwarp();
        if (lane == 0) { red[0][0] = a; red[0][1] = b; red[0][2] = c; }
    }
    __syncthreads();
    x = red[0][0]; y = red[0][1]; z = red[0][2];
    __syncthreads();
}

// S0 = sum e_i, S1 = sum e_i D_i, S2 = sum e_i D_i^2 over the finite costs,
// D_i = C_min - C_i, e_i = exp(D_i / eta)
// (FP32 exponentials, FP64 sums, for the search; FP64 throughout for the
// final step)
template <bool FP32_EXP>
__device__ void reps_sums(const OptArgs &a, double cmin, double inv_eta, double &S0, double &S1, double &S2,
                          double (*red)[3]) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < a.N; i += kSoft) {
        const double c = a.c_mean[i];
        if (!isfinite(c)) continue;
        const double d = cmin - c;
        const double e = FP32_EXP ? (double)__expf((float)(d * inv_eta)) : exp(d * inv_eta);
        s0 += e; s1 += e * d; s2 += e * d * d;
    }
    block_sum3(s0, s1, s2, red);
    S0 = s0; S1 = s1; S2 = s2;
}

// One CTA: C_min, C_max and the number K of finite window means, i*, the REPS
// temperature, the weights and their inclusive CDF in index order (elite_w),
// the total (misc[M_WSUM]).
__global__ void __launch_bounds__(kSoft) soft_weights_kernel(const OptArgs a) {
    __shared__ double red[kSoft / 32][3];
    __shared__ unsigned long long s_min_key;
    __shared__ int s_min_idx;
    const int N = a.N, t = threadIdx.x;
    double lo = INFINITY, hi = -INFINITY, cnt = 0.0;
    unsigned long long bk = ~0ull;
    int bi = 0x7fffffff;
    for (int i = t; i < N; i += kSoft) {
        const double c = a.c_mean[i];
        if (isfinite(c)) { lo = fmin(lo, c); hi = fmax(hi, c); cnt += 1.0; }
        const unsigned long long key = order_key(c);
        if (key < bk || (key == bk && i < bi)) { bk = key; bi = i; }
    }
    // min and max as sums of one-hot terms would be inexact: reduce them directly
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ok < bk || (ok == bk && oi < bi)) { bk = ok; bi = oi; }
    }
    if (t == 0) { s_min_key = ~0ull; s_min_idx = 0x7fffffff; }
    if ((t & 31) == 0) { red[t >> 5][0] = lo; red[t >> 5][1] = hi; red[t >> 5][2] = cnt; }
    __syncthreads();
    if ((t & 31) == 0) atomicMin(&s_min_key, bk);
    if (t < 32) {   // the first warp combines the warps' partials
        double mn = red[t][0], mx = red[t][1], ct = red[t][2];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            ct += __shfl_xor_sync(0xffffffffu, ct, o);
        }
        __syncwarp();
        if (t == 0) { red[0][0] = mn; red[0][1] = mx; red[0][2] = ct; }
    }
    __syncthreads();
    const double cmin = red[0][0], cmax = red[0][1], K = red[0][2];
    __syncthreads();
    if ((t & 31) == 0 && bk == s_min_key) atomicMin(&s_min_idx, bi);
    double nmin = 0.0;
    for (int i = t; i < N; i += kSoft) nmin += (a.c_mean[i] == cmin) ? 1.0 : 0.0;
    double z0 = 0.0, z1 = 0.0;
    block_sum3(nmin, z0, z1, red);
    const int istar = s_min_idx;

    // REPS temperature: the root of g'(eta) = eps + log(S0/K) - S1/(eta S0) by
    // Newton steps in t = log(eta) (dg'/dt = Var_w(D)/eta^2) inside a
    // shrinking bracket, bisecting when a step leaves it
    double eta = NAN;
    if (a.kind == 2 && K > 0.0) {
        const double eps = a.reps_epsilon;
        if (!(cmax > cmin)) {
            eta = INFINITY;
        } else if (eps >= log(K / nmin)) {
            eta = 0.0;
        } else {
            // the scalar steps run in thread 0 and reach the block through
            // shared memory (FP64 transcendentals are costly on this part)
            __shared__ double s_sc[4];   // e^t, 1/e^t, t, done flag
            double S0, S1, S2;
            double tlo = 0.0, thi = 0.0, tt = 0.0;
            if (t == 0) {
                const double lr = log(cmax - cmin);
                tlo = lr - 50.0;
                thi = lr + 50.0;
                s_sc[0] = exp(tlo); s_sc[1] = 1.0 / s_sc[0];
            }
            __syncthreads();
            for (int k = 0; k < 200; ++k) {   // widen the bracket until g'(e^tlo) < 0 (a sign: FP32 will do)
                reps_sums<true>(a, cmin, s_sc[1], S0, S1, S2, red);
                if (t == 0) {
                    const bool below = eps + log(S0 / K) - S1 / (s_sc[0] * S0) < 0.0;
                    if (!below) { tlo -= 50.0; s_sc[0] = exp(tlo); s_sc[1] = 1.0 / s_sc[0]; }
                    s_sc[3] = below ? 1.0 : 0.0;
                }
                __syncthreads();
                const bool done = s_sc[3] != 0.0;
                __syncthreads();
                if (done) break;
            }
            if (t == 0) { tt = 0.5 * (tlo + thi); s_sc[0] = exp(tt); s_sc[1] = 1.0 / s_sc[0]; s_sc[2] = tt; s_sc[3] = 0.0; }
            __syncthreads();
            // Newton steps with FP32 exponentials down to FP32 accuracy, then
            // one step with FP64 sums: Newton's quadratic convergence takes
            // the ~1e-7 error of the FP32 root to ~1e-14
            for (int it = 0; it < 201; ++it) {
                const bool last = s_sc[3] == 2.0;
                if (last) reps_sums<false>(a, cmin, s_sc[1], S0, S1, S2, red);
                else reps_sums<true>(a, cmin, s_sc[1], S0, S1, S2, red);
                if (t == 0) {
                    const double e = s_sc[0];
                    const double g1 = eps + log(S0 / K) - S1 / (e * S0);
                    if (g1 < 0.0) tlo = tt; else thi = tt;
                    const double mean = S1 / S0, var = S2 / S0 - mean * mean;
                    const double slope = var / (e * e);
                    double tn = (slope > 0.0) ? tt - g1 / slope : 0.5 * (tlo + thi);
                    if (!(tn > tlo && tn < thi)) tn = 0.5 * (tlo + thi);
                    const bool near = fabs(tn - tt) <= 1e-6 * (1.0 + fabs(tt)) || thi - tlo <= 1e-6 * (1.0 + fabs(tt));
                    tt = tn;
                    s_sc[0] = exp(tt); s_sc[1] = 1.0 / s_sc[0]; s_sc[2] = tt;
                    s_sc[3] = last ? 1.0 : (near || it == 199 ? 2.0 : 0.0);
                }
                __syncthreads();
                const bool done = s_sc[3] == 1.0;
                __syncthreads();
                if (done) break;
            }
            eta = s_sc[0];
        }
    }
    if (t == 0) {   // for the weights (grid) and the CDF
        a.misc[M_U] = eta;
        a.misc[M_CMIN] = cmin;
        a.misc[M_NFIN] = K;
        a.misc[M_ISTAR] = (double)istar;
        *a.argmin_state = istar;
        if (a.argmin_out) *a.argmin_out = istar;
    }
}

// One thread per environment: its weight (FP64), into elite_w.
__global__ void soft_w_kernel(const OptArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const double eta = a.misc[M_U], cmin = a.misc[M_CMIN], K = a.misc[M_NFIN];
    const double c = a.c_mean[i];
    double w;
    if (K == 0.0) w = 1.0;
    else if (!isfinite(c)) w = 0.0;
    else if (a.kind == 1) w = exp(-a.wrs_lambda * (c - cmin));
    else if (isinf(eta)) w = 1.0;
    else if (eta == 0.0) w = (c == cmin) ? 1.0 : 0.0;
    else w = exp((cmin - c) / eta);
    a.elite_w[i] = w;
}

// One CTA: the inclusive CDF of the weights in index order (chunks of kSoft,
// carried), in place, and the total (misc[M_WSUM]).
__global__ void __launch_bounds__(kSoft) soft_cdf_kernel(const OptArgs a) {
    __shared__ double red[kSoft / 32][3];
    const int N = a.N, t = threadIdx.x;
    double carry = 0.0;
    const int lane = t & 31, wid = t >> 5;
    for (int base = 0; base < N; base += kSoft) {
        const int i = base + t;
        const double w = (i < N) ? a.elite_w[i] : 0.0;
        double inc = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) red[wid][0] = inc;
        __syncthreads();
        if (wid == 0) {   // exclusive scan of the warps' totals by the first warp
            const double v = red[lane][0];
            double x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double u = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += u;
            }
            __syncwarp();
            red[lane][1] = x - v;
            if (lane == 31) red[0][2] = x;
        }
        __syncthreads();
        if (i < N) a.elite_w[i] = carry + (red[wid][1] + inc);
        carry += red[0][2];
        __syncthreads();
    }
    if (t == 0) a.misc[M_WSUM] = carry;
}

// Four lanes per environment: lane 0 draws the parent (inverse CDF), every
// lane one Box-Muller pair of the exploration noise; lane 0 writes the state.
__global__ void __launch_bounds__(kOptBlock * kApplyLanes) soft_apply_kernel(const OptArgs a) {
    const int sub = threadIdx.x & (kApplyLanes - 1);
    const int i = blockIdx.x * kOptBlock + (int)(threadIdx.x / kApplyLanes);
    const unsigned qmask = 0xfu << (threadIdx.x & 28u);
    const int N = a.N;
    if (i >= N) return;   // whole quads
    const uint32_t upd = a.win ? a.win->update_index : a.update_index;
    int par = 0;
    if (sub == 0) {
        if (i == 0) *a.n_window = 0;
        a.c_sum[i] = 0.0;
        if (a.cache_n) a.cache_n[i] = 0;   // replaced: its solver starts cold
        const uint4 uw = rng_words(a.seed, 3, upd, (uint32_t)i, 0);
        const double pos = unit53(uw.x, uw.y) * a.misc[M_WSUM];
        int lo = 0, hi = N - 1;   // first j with pos < CDF_j
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (pos < a.elite_w[mid]) hi = mid; else lo = mid + 1;
        }
        par = lo;
        if (a.parent_out) a.parent_out[i] = par;
    }
    double e0, e1;
    gauss2(rng_words(a.seed, 1, upd, (uint32_t)i, (uint32_t)sub), e0, e1);
    double eps[8];
#pragma unroll
    for (int b = 0; b < kApplyLanes; ++b) {
        eps[2 * b] = __shfl_sync(qmask, e0, b, kApplyLanes);
        eps[2 * b + 1] = __shfl_sync(qmask, e1, b, kApplyLanes);
    }
    if (sub != 0) return;
    const float4 p0 = a.sn_pose[2 * par], p1 = a.sn_pose[2 * par + 1];
    float4 v0 = a.sn_vel[2 * par], v1 = a.sn_vel[2 * par + 1];
    if (a.explore_velocity) {
        a.pose[2 * i] = p0;
        a.pose[2 * i + 1] = p1;
        v0 = make_float4((float)(v0.x + (double)a.sigma_vel[0] * eps[0]), (float)(v0.y + (double)a.sigma_vel[1] * eps[1]),
                         (float)(v0.z + (double)a.sigma_vel[2] * eps[2]), 0.0f);
        v1 = make_float4((float)(v1.x + (double)a.sigma_vel[3] * eps[3]), (float)(v1.y + (double)a.sigma_vel[4] * eps[4]),
                         (float)(v1.z + (double)a.sigma_vel[5] * eps[5]), 0.0f);
    } else {
        const Q4d qn = qnorm_d(qmul_d(qexp_d((double)a.sigma_pose[3] * eps[3], (double)a.sigma_pose[4] * eps[4],
                                             (double)a.sigma_pose[5] * eps[5]),
                                      {p1.x, p1.y, p1.z, p1.w}));
        a.pose[2 * i] = make_float4((float)(p0.x + (double)a.sigma_pose[0] * eps[0]),
                                    (float)(p0.y + (double)a.sigma_pose[1] * eps[1]),
                                    (float)(p0.z + (double)a.sigma_pose[2] * eps[2]), 0.0f);
        a.pose[2 * i + 1] = make_float4((float)qn.w, (float)qn.x, (float)qn.y, (float)qn.z);
    }
    a.vel[2 * i] = v0;
    a.vel[2 * i + 1] = v1;
    const float2 th = a.sn_params[par];
    const double m = fmin(fmax((double)th.x + (double)a.sigma_theta[0] * eps[6], (double)a.m_lo), (double)a.m_hi);
    const double mu = fmin(fmax((double)th.y + (double)a.sigma_theta[1] * eps[7], (double)a.mu_lo), (double)a.mu_hi);
    a.params[i] = make_float2((float)m, (float)mu);
    a.status[i] = a.sn_status[par];
    if (a.qj) {   // the parent's hand, from the snapshot
        const int D = a.D;
        for (int j = 0; j < D; ++j) {
            a.qj[(size_t)i * D + j] = a.sn_qj[(size_t)par * D + j];
            a.qdj[(size_t)i * D + j] = a.sn_qdj[(size_t)par * D + j];
        }
    }
}

__global__ void win_desc_kernel(WinDesc *d, WinDesc v) { *d = v; }

}  // namespace

cudaError_t launch_win_desc(WinDesc *d, WinDesc v, cudaStream_t s) {
    win_desc_kernel<<<1, 1, 0, s>>>(d, v);
    return cudaGetLastError();
}

int opt_blocks(int N) { return (N + kOptBlock - 1) / kOptBlock; }

cudaError_t launch_select(const OptArgs &a, cudaStream_t s) {
    if (a.N <= kKeys * kSelSmall) select_kernel<kSelSmall><<<1, kSelSmall, 0, s>>>(a);
    else select_kernel<kSel><<<1, kSel, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_optimizer(const OptArgs &a, cudaStream_t s) {
    if (a.kind != 0) {   // WRS / REPS: weights, snapshot of the state, draws and exploration
        const size_t N = a.N;
        soft_weights_kernel<<<1, kSoft, 0, s>>>(a);
        soft_w_kernel<<<(a.N + 127) / 128, 128, 0, s>>>(a);
        soft_cdf_kernel<<<1, kSoft, 0, s>>>(a);
        cudaError_t e = cudaMemcpyAsync(a.sn_pose, a.pose, 2 * N * sizeof(float4), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(a.sn_vel, a.vel, 2 * N * sizeof(float4), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(a.sn_params, a.params, N * sizeof(float2), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(a.sn_status, a.status, N * sizeof(int), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && a.qj) {
            const size_t hb = N * (size_t)a.D * sizeof(float);
            e = cudaMemcpyAsync(a.sn_qj, a.qj, hb, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(a.sn_qdj, a.qdj, hb, cudaMemcpyDeviceToDevice, s);
        }
        if (e != cudaSuccess) return e;
        soft_apply_kernel<<<opt_blocks(a.N), kOptBlock * kApplyLanes, 0, s>>>(a);
        return cudaGetLastError();
    }
    // the elite count, computed exactly as select_kernel does
    int k = (int)floor((double)a.elite_frac * (double)a.N);
    k = k < 1 ? 1 : (k > a.N ? a.N : k);
    const int kb = opt_blocks(k), nb = opt_blocks(a.N);
    cudaError_t e = a.N <= kKeys * kSelSmall ? launch_dependent(select_kernel<kSelSmall>, 1, kSelSmall, s, a)
                                             : launch_dependent(select_kernel<kSel>, 1, kSel, s, a);
    if (e == cudaSuccess) e = launch_dependent(stats_kernel, kb, kOptBlock * kStatWarps, s, a);
    if (e == cudaSuccess) e = launch_dependent(finalize_kernel, 1, kFin, s, a, kb);
    if (e == cudaSuccess) e = launch_dependent(apply_kernel, nb, kOptBlock * kApplyLanes, s, a);
    return e;
}

}  // namespace ih
