// Krylov vector kernels of the GMRES core (Sec. 3.2): modified Gram-Schmidt
// steps (w -= h_k v_k fused with the next projection <w, v_{k+1}>, or with
// ||w||^2 after the last one), the first projection <w, v_0> and norms, the
// solution update x += sum y_i z_i and scalings.
//
// These are streaming kernels over packed Stokes vectors of N doubles.  The
// number of basis vectors of an update is a template parameter (dispatched
// at run time), loads are 16-byte, the grid is a function of the vector
// length alone (about four pairs of values per thread, at most KRY_BLOCKS
// blocks = 8 per SM; kry_blocks) and every reduction sums its block partials
// in a fixed order, so results are bitwise reproducible.  On GB300 the FP64
// FMA rate (about 1.2 TFLOP/s) caps a pass at about one FMA per 8 bytes
// read; the passes that only read issue the loads of LOOKAHEAD steps before
// their FMAs, so that a thread's chain of dependent FMAs does not also wait
// for one load at a time.
#include "internal.cuh"

namespace stk {
namespace {

constexpr int KT = 256;
constexpr int MAXV = 33;

struct PtrArr {
    const void* p[MAXV];
};

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Reduce NV per-thread values over the block; value i of block b goes to
// part[i * stride + b].
template <int NV>
__device__ __forceinline__ void block_sums(const double (&v)[NV], double* part, int stride) {
    __shared__ double sh[NV][KT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double s = wsum(v[i]);
        if (lane == 0) sh[i][w] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < KT / 32; ++k) s += sh[threadIdx.x][k];
        part[threadIdx.x * stride + blockIdx.x] = s;
    }
}

// The final sums of a reduction, done by the block that finishes last
// instead of by a launch of their own.  Every block has written its NV
// partials at part[k * nb + b] (nb = gridDim.x blocks; a stacked batch
// counts per instance, blockIdx.y).  The block whose arrival completes the
// count *cnt forms out[k] = sum_b part[k * nb + b] for each k in a fixed
// order (thread t adds b = t, t + KT, ..., then a shuffle tree per warp and
// the warps' sums in order) and resets the count for the next reduction on
// the stream (kernels on a stream never overlap: each waits at pdl_entry()
// for its predecessor to complete).  Returns true in that block, whose
// thread 0 wrote every out[k].
template <int NV>
__device__ __forceinline__ bool finish_last(const double* part, int nb, double* out, unsigned* cnt) {
    __shared__ unsigned s_last;
    __shared__ double sh[KT / 32];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(cnt, 1u) == gridDim.x - 1u ? 1u : 0u;
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    for (int k = 0; k < NV; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nb; b += KT) s += __ldcg(part + (size_t)k * nb + b);
        s = wsum(s);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double r = 0.0;
#pragma unroll
            for (int i = 0; i < KT / 32; ++i) r += sh[i];
            out[k] = r;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *cnt = 0u;
    return true;
}

// Number of grid-stride steps whose loads a read-only pass issues before
// using any of them (its adds keep the order of the steps).
constexpr int LOOKAHEAD = 4;

// The partial sums of pass J of thread pair index t, stride st, over the
// pairs t < n2: acc[i] += <w, V_i> (i <= J), or acc[0] += <w, w> for J = -1,
// pair after pair.  `pair(t)` maps a step to its pair of values.
template <int J, typename PairOf>
__device__ __forceinline__ void dot_pass(const PtrArr& V, const double2* __restrict__ w2, int t, int n2,
                                         int st, PairOf pair, double (&acc)[J >= 0 ? J + 1 : 1]) {
    for (; t < n2 - (LOOKAHEAD - 1) * st; t += LOOKAHEAD * st) {
        int p[LOOKAHEAD];
        double2 a[LOOKAHEAD];
#pragma unroll
        for (int u = 0; u < LOOKAHEAD; ++u) {
            p[u] = pair(t + u * st);
            a[u] = w2[p[u]];
        }
        if constexpr (J < 0) {
#pragma unroll
            for (int u = 0; u < LOOKAHEAD; ++u) {
                acc[0] = fma(a[u].x, a[u].x, acc[0]);
                acc[0] = fma(a[u].y, a[u].y, acc[0]);
            }
        } else {
#pragma unroll
            for (int i = 0; i <= J; ++i) {
                double2 v[LOOKAHEAD];
#pragma unroll
                for (int u = 0; u < LOOKAHEAD; ++u) v[u] = reinterpret_cast<const double2*>(V.p[i])[p[u]];
#pragma unroll
                for (int u = 0; u < LOOKAHEAD; ++u) {
                    acc[i] = fma(a[u].x, v[u].x, acc[i]);
                    acc[i] = fma(a[u].y, v[u].y, acc[i]);
                }
            }
        }
    }
    for (; t < n2; t += st) {
        const int p = pair(t);
        const double2 a = w2[p];
        if constexpr (J < 0) {
            acc[0] = fma(a.x, a.x, acc[0]);
            acc[0] = fma(a.y, a.y, acc[0]);
        } else {
#pragma unroll
            for (int i = 0; i <= J; ++i) {
                const double2 v = reinterpret_cast<const double2*>(V.p[i])[p];
                acc[i] = fma(a.x, v.x, acc[i]);
                acc[i] = fma(a.y, v.y, acc[i]);
            }
        }
    }
}

// The sum over the float4 steps i, i + st, ... < n4 of each step's four
// values (summed in FP32 in pairs, widened once), step after step.
__device__ __forceinline__ double sum4_pass(const float4* __restrict__ x4, int i, int n4, int st) {
    double s = 0.0;
    for (; i < n4 - (LOOKAHEAD - 1) * st; i += LOOKAHEAD * st) {
        float4 v[LOOKAHEAD];
#pragma unroll
        for (int u = 0; u < LOOKAHEAD; ++u) v[u] = x4[i + u * st];
#pragma unroll
        for (int u = 0; u < LOOKAHEAD; ++u) s += double((v[u].x + v[u].y) + (v[u].z + v[u].w));
    }
    for (; i < n4; i += st) {
        const float4 v = x4[i];
        s += double((v.x + v.y) + (v.z + v.w));
    }
    return s;
}

// h[i] = <w, V_i> (i <= J); for J = -1, h[0] = <w, w>
template <int J>
__global__ void __launch_bounds__(KT) k_mdot(int n, PtrArr V, const double* __restrict__ w,
                                              double* __restrict__ part, double* out, unsigned* cnt) {
    constexpr int NV = J >= 0 ? J + 1 : 1;
    pdl_entry();
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    dot_pass<J>(V, reinterpret_cast<const double2*>(w), blockIdx.x * KT + threadIdx.x, n >> 1, gridDim.x * KT,
                [](int t) { return t; }, acc);
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const double a = w[n - 1];
        if constexpr (J < 0) {
            acc[0] = fma(a, a, acc[0]);
        } else {
#pragma unroll
            for (int i = 0; i <= J; ++i) acc[i] = fma(a, static_cast<const double*>(V.p[i])[n - 1], acc[i]);
        }
    }
    block_sums<NV>(acc, part, gridDim.x);
    finish_last<NV>(part, gridDim.x, out, cnt);
}

// One modified Gram-Schmidt step: w -= h[k] v_k, then the block partials
// of <w, u> (u = v_{k+1}), or of <w, w> when u is null.
__global__ void __launch_bounds__(KT) k_mgs_step(int n, const double* __restrict__ vk,
                                                 const double* __restrict__ u,
                                                 const double* __restrict__ h, int k,
                                                 double* __restrict__ w, double* __restrict__ part,
                                                 double* out, unsigned* cnt) {
    pdl_entry();
    const double hk = h[k];
    double s[1] = {0.0};
    const int n2 = n >> 1;
    double2* w2 = reinterpret_cast<double2*>(w);
    const double2* v2 = reinterpret_cast<const double2*>(vk);
    const double2* u2 = reinterpret_cast<const double2*>(u);
    for (int t = blockIdx.x * KT + threadIdx.x; t < n2; t += gridDim.x * KT) {
        double2 a = w2[t];
        const double2 v = v2[t];
        a.x = fma(-hk, v.x, a.x);
        a.y = fma(-hk, v.y, a.y);
        w2[t] = a;
        const double2 b = u ? u2[t] : a;
        s[0] = fma(a.x, b.x, s[0]);
        s[0] = fma(a.y, b.y, s[0]);
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        double a = fma(-hk, vk[n - 1], w[n - 1]);
        w[n - 1] = a;
        s[0] = fma(a, u ? u[n - 1] : a, s[0]);
    }
    block_sums<1>(s, part, gridDim.x);
    finish_last<1>(part, gridDim.x, out, cnt);
}

template <typename TV> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

// x += sum_{i < K} y[i] V_i
template <int K, typename TV>
__global__ void __launch_bounds__(KT) k_comb(int n, PtrArr V, const double* __restrict__ y,
                                              double* __restrict__ x) {
    pdl_entry();
    using V2 = typename Vec2<TV>::type;
    double yy[K];
#pragma unroll
    for (int i = 0; i < K; ++i) yy[i] = y[i];
    const int n2 = n >> 1;
    double2* x2 = reinterpret_cast<double2*>(x);
    for (int t = blockIdx.x * KT + threadIdx.x; t < n2; t += gridDim.x * KT) {
        double2 a = x2[t];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const V2 v = reinterpret_cast<const V2*>(V.p[i])[t];
            a.x = fma(yy[i], widen(v.x), a.x);
            a.y = fma(yy[i], widen(v.y), a.y);
        }
        x2[t] = a;
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        double a = x[n - 1];
#pragma unroll
        for (int i = 0; i < K; ++i) a = fma(yy[i], widen(static_cast<const TV*>(V.p[i])[n - 1]), a);
        x[n - 1] = a;
    }
}

// x += sum_{i < *k} y[i] V_i with *k <= K read on the device (the branch is
// uniform: the vectors beyond *k are not loaded)
template <int K, typename TV>
__global__ void __launch_bounds__(KT) k_comb_dev(int n, PtrArr V, const double* __restrict__ y,
                                                  const int* __restrict__ kp, double* __restrict__ x) {
    pdl_entry();
    using V2 = typename Vec2<TV>::type;
    const int k = *kp;
    if (k <= 0) return;
    double yy[K];
#pragma unroll
    for (int i = 0; i < K; ++i) yy[i] = i < k ? y[i] : 0.0;
    const int n2 = n >> 1;
    double2* x2 = reinterpret_cast<double2*>(x);
    for (int t = blockIdx.x * KT + threadIdx.x; t < n2; t += gridDim.x * KT) {
        double2 a = x2[t];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            if (i < k) {
                const V2 v = reinterpret_cast<const V2*>(V.p[i])[t];
                a.x = fma(yy[i], widen(v.x), a.x);
                a.y = fma(yy[i], widen(v.y), a.y);
            }
        }
        x2[t] = a;
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        double a = x[n - 1];
#pragma unroll
        for (int i = 0; i < K; ++i)
            if (i < k) a = fma(yy[i], widen(static_cast<const TV*>(V.p[i])[n - 1]), a);
        x[n - 1] = a;
    }
}

__global__ void __launch_bounds__(KT) k_scal(int n, double* __restrict__ x, double a,
                                             const double* __restrict__ nrm2) {
    pdl_entry();
    const double s = nrm2 ? 1.0 / sqrt(*nrm2) : a;
    for (int t = blockIdx.x * KT + threadIdx.x; t < n; t += gridDim.x * KT) x[t] *= s;
}

// ------------------------------------------------------------ stacked batches
// The kernels above on every instance of a stacked batch at once (grid
// (nbu, nsl), blockIdx.y the instance).  Instance y's values are visited in
// the order of its own packed vector (sl_pair), with the partition over
// threads and the summation order of the single-instance kernels (the same
// grid per instance, kry_blocks, and the final sums per instance in its last
// block), so its projections, norms and updates are bitwise the ones it gets
// alone.

// global pair index of pair t (values 2t, 2t + 1) of instance y
__device__ __forceinline__ int sl_pair(const SliceMap& m, int y, int t) {
    int i = 2 * t;
    if (i < m.len[0]) return (m.off[0] + y * m.len[0] + i) >> 1;
    i -= m.len[0];
    if (i < m.len[1]) return (m.off[1] + y * m.len[1] + i) >> 1;
    i -= m.len[1];
    return (m.off[2] + y * m.len[2] + i) >> 1;
}

template <int J>
__global__ void __launch_bounds__(KT) k_mdot_sl(SliceMap m, PtrArr V, const double* __restrict__ w,
                                                 double* __restrict__ part, double* out, int ostride,
                                                 unsigned* cnt) {
    constexpr int NV = J >= 0 ? J + 1 : 1;
    const int nbu = gridDim.x;
    pdl_entry();
    const int y = blockIdx.y;
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    dot_pass<J>(V, reinterpret_cast<const double2*>(w), blockIdx.x * KT + threadIdx.x, m.nl >> 1,
                gridDim.x * KT, [&m, y](int t) { return sl_pair(m, y, t); }, acc);
    block_sums<NV>(acc, part + (size_t)y * NV * nbu, nbu);
    finish_last<NV>(part + (size_t)y * NV * nbu, nbu, out + (size_t)y * ostride, cnt + y);
}

__global__ void __launch_bounds__(KT) k_mgs_step_sl(SliceMap m, const double* __restrict__ vk,
                                                    const double* __restrict__ u,
                                                    const double* __restrict__ h, int hstride, int k,
                                                    double* __restrict__ w, double* __restrict__ part,
                                                    double* out, int ostride, unsigned* cnt) {
    pdl_entry();
    const int nbu = gridDim.x;
    const int y = blockIdx.y;
    const double hk = h[(size_t)y * hstride + k];
    double s[1] = {0.0};
    const int n2 = m.nl >> 1;
    double2* w2 = reinterpret_cast<double2*>(w);
    const double2* v2 = reinterpret_cast<const double2*>(vk);
    const double2* u2 = reinterpret_cast<const double2*>(u);
    for (int t = blockIdx.x * KT + threadIdx.x; t < n2; t += gridDim.x * KT) {
        const int p = sl_pair(m, y, t);
        double2 a = w2[p];
        const double2 v = v2[p];
        a.x = fma(-hk, v.x, a.x);
        a.y = fma(-hk, v.y, a.y);
        w2[p] = a;
        const double2 b = u ? u2[p] : a;
        s[0] = fma(a.x, b.x, s[0]);
        s[0] = fma(a.y, b.y, s[0]);
    }
    block_sums<1>(s, part + (size_t)y * nbu, nbu);
    finish_last<1>(part + (size_t)y * nbu, nbu, out + (size_t)y * ostride, cnt + y);
}

// x += sum_{i < k_y} y_y[i] V_i with k_y, y_y from instance y's GMRES state
template <int K, typename TV>
__global__ void __launch_bounds__(KT) k_comb_dev_sl(SliceMap m, PtrArr V, const GmState* __restrict__ st,
                                                     double* __restrict__ x) {
    pdl_entry();
    using V2 = typename Vec2<TV>::type;
    const GmState& S = st[blockIdx.y];
    const int k = S.k;
    if (k <= 0) return;
    double yy[K];
#pragma unroll
    for (int i = 0; i < K; ++i) yy[i] = i < k ? S.y[i] : 0.0;
    const int n2 = m.nl >> 1;
    double2* x2 = reinterpret_cast<double2*>(x);
    for (int t = blockIdx.x * KT + threadIdx.x; t < n2; t += gridDim.x * KT) {
        const int p = sl_pair(m, blockIdx.y, t);
        double2 a = x2[p];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            if (i < k) {
                const V2 v = reinterpret_cast<const V2*>(V.p[i])[p];
                a.x = fma(yy[i], widen(v.x), a.x);
                a.y = fma(yy[i], widen(v.y), a.y);
            }
        }
        x2[p] = a;
    }
}

// Arnoldi step j's basis vector: x *= inv_scale of instance y where step j
// is open; zero where it is not (an instance that has stopped carries zeros
// through the rest of the cycle, so its vectors stay finite).
__global__ void __launch_bounds__(KT) k_scal_dev_sl(SliceMap m, double* __restrict__ x,
                                                    const GmState* __restrict__ st, int j) {
    pdl_entry();
    const GmState& S = st[blockIdx.y];
    const bool open = S.cond[GM_COND_STEP0 + j] != 0;
    const double a = S.inv_scale;
    const int n2 = m.nl >> 1;
    double2* x2 = reinterpret_cast<double2*>(x);
    for (int t = blockIdx.x * KT + threadIdx.x; t < n2; t += gridDim.x * KT) {
        const int p = sl_pair(m, blockIdx.y, t);
        double2 v = x2[p];
        v.x = open ? v.x * a : 0.0;
        v.y = open ? v.y * a : 0.0;
        x2[p] = v;
    }
}

// per-instance k_sum_f32x4 (instances of n values one after another):
// out[y * ostride] = the sum of instance y, out[y * ostride + 1] its mean
__global__ void __launch_bounds__(KT) k_sum_f32x4_sl(int n, const float* __restrict__ x, double* part,
                                                     double* out, int ostride, unsigned* cnt) {
    pdl_entry();
    const int nbu = gridDim.x;
    const float* xs = x + (size_t)blockIdx.y * n;
    const int n4 = n >> 2;
    const float4* x4 = reinterpret_cast<const float4*>(xs);
    double acc[1] = {sum4_pass(x4, blockIdx.x * KT + threadIdx.x, n4, gridDim.x * KT)};
    if (blockIdx.x == 0 && threadIdx.x < (n & 3)) acc[0] += double(xs[4 * n4 + threadIdx.x]);
    block_sums<1>(acc, part + (size_t)blockIdx.y * nbu, nbu);
    double* o = out + (size_t)blockIdx.y * ostride;
    if (finish_last<1>(part + (size_t)blockIdx.y * nbu, nbu, o, cnt + blockIdx.y) && threadIdx.x == 0)
        o[1] = o[0] / n;
}

// Blocks of a pass over `items` loads (pairs of doubles, or float4): about
// four per thread, at most KRY_BLOCKS.  A function of one instance's vector
// length alone, so a stacked batch partitions each instance exactly as a
// single handle does.  (A fixed KRY_BLOCKS grid left most threads of a
// small vector with one load or none and made per-block overhead the cost.)
int kry_blocks(int items) {
    constexpr int PER_THREAD = 4;
    const int b = (items + KT * PER_THREAD - 1) / (KT * PER_THREAD);
    return b < 1 ? 1 : (b > KRY_BLOCKS ? KRY_BLOCKS : b);
}

PtrArr pack(const void* const* V, int k) {
    PtrArr pa{};
    for (int i = 0; i < k; ++i) pa.p[i] = V[i];
    return pa;
}

// Partial sums of an FP32 vector (n % 4 == 0 handled by block 0's tail,
// x 16-byte aligned): four elements per 16-byte load, summed in FP32 in a
// fixed order and widened to FP64 once per four.  The widening runs on
// GB300's FP64 pipe, so one per element made this pass FP64-bound; the
// FP32 sum of four adds a relative rounding of about 2^-23 to each term,
// below the FP32 data's own.
__global__ void __launch_bounds__(KT) k_sum_f32x4(int n, const float* __restrict__ x, double* part,
                                                   double* out, unsigned* cnt) {
    pdl_entry();
    const int n4 = n >> 2;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    double acc[1] = {sum4_pass(x4, blockIdx.x * KT + threadIdx.x, n4, gridDim.x * KT)};
    if (blockIdx.x == 0 && threadIdx.x < (n & 3)) acc[0] += double(x[4 * n4 + threadIdx.x]);
    block_sums<1>(acc, part, gridDim.x);
    if (finish_last<1>(part, gridDim.x, out, cnt) && threadIdx.x == 0) out[1] = out[0] / n;
}

}  // namespace

void launch_sum_f32x4(int n, const float* x, double* scratch, double* out, unsigned* cnt, cudaStream_t s) {
    launch_pdl(k_sum_f32x4, dim3(kry_blocks(n >> 2)), dim3(KT), s, n, x, scratch, out, cnt);
}

#define STK_J_CASES(X) \
    X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) \
    X(16) X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30) X(31)

void launch_multidot(int n, int j, const double* const* V, const double* w, double* scratch,
                     double* h, unsigned* cnt, cudaStream_t s) {
    PtrArr pa = pack(reinterpret_cast<const void* const*>(V), j < 0 ? 0 : 1);
    const int nb = kry_blocks(n >> 1);
    if (j < 0) launch_pdl(k_mdot<-1>, dim3(nb), dim3(KT), s, n, pa, w, scratch, h, cnt);
    else launch_pdl(k_mdot<0>, dim3(nb), dim3(KT), s, n, pa, w, scratch, h, cnt);
}

template <typename TV>
void launch_combine(int n, int k, const TV* const* V, const double* y, double* x, cudaStream_t s) {
    PtrArr pa = pack(reinterpret_cast<const void* const*>(V), k);
    switch (k - 1) {
#define X(J) case J: launch_pdl(k_comb<J + 1, TV>, dim3(kry_blocks(n >> 1)), dim3(KT), s, n, pa, y, x); break;
    STK_J_CASES(X)
#undef X
    default: return;
    }
}

template <typename TV>
void launch_combine_dev(int n, int m, const TV* const* V, const double* y, const int* k, double* x,
                        cudaStream_t s) {
    PtrArr pa = pack(reinterpret_cast<const void* const*>(V), m);
    switch (m - 1) {
#define X(J) case J: launch_pdl(k_comb_dev<J + 1, TV>, dim3(kry_blocks(n >> 1)), dim3(KT), s, n, pa, y, k, x); break;
    STK_J_CASES(X)
#undef X
    default: return;
    }
}

void launch_mgs_step(int n, const double* vk, const double* u, const double* h, int k, double* w,
                     double* scratch, double* out, unsigned* cnt, cudaStream_t s) {
    launch_pdl(k_mgs_step, dim3(kry_blocks(n >> 1)), dim3(KT), s, n, vk, u, h, k, w, scratch, out, cnt);
}

void launch_sum_f32x4_sl(int n, int nsl, const float* x, double* scratch, double* out, int ostride,
                         unsigned* cnt, cudaStream_t s) {
    launch_pdl(k_sum_f32x4_sl, dim3(kry_blocks(n >> 2), nsl), dim3(KT), s, n, x, scratch, out, ostride, cnt);
}

void launch_multidot_sl(const SliceMap& m, int nsl, int j, const double* const* V, const double* w,
                        double* scratch, double* h, int hstride, unsigned* cnt, cudaStream_t s) {
    PtrArr pa = pack(reinterpret_cast<const void* const*>(V), j < 0 ? 0 : 1);
    const dim3 gr(kry_blocks(m.nl >> 1), nsl);
    if (j < 0) launch_pdl(k_mdot_sl<-1>, gr, dim3(KT), s, m, pa, w, scratch, h, hstride, cnt);
    else launch_pdl(k_mdot_sl<0>, gr, dim3(KT), s, m, pa, w, scratch, h, hstride, cnt);
}

void launch_mgs_step_sl(const SliceMap& m, int nsl, const double* vk, const double* u, const double* h,
                        int hstride, int k, double* w, double* scratch, double* out, int ostride,
                        unsigned* cnt, cudaStream_t s) {
    launch_pdl(k_mgs_step_sl, dim3(kry_blocks(m.nl >> 1), nsl), dim3(KT), s, m, vk, u, h, hstride, k, w,
               scratch, out, ostride, cnt);
}

template <typename TV>
void launch_combine_dev_sl(const SliceMap& m, int nsl, int mmax, const TV* const* V, const GmState* st,
                           double* x, cudaStream_t s) {
    PtrArr pa = pack(reinterpret_cast<const void* const*>(V), mmax);
    const dim3 gr(kry_blocks(m.nl >> 1), nsl);
    switch (mmax - 1) {
#define X(J) case J: launch_pdl(k_comb_dev_sl<J + 1, TV>, gr, dim3(KT), s, m, pa, st, x); break;
    STK_J_CASES(X)
#undef X
    default: return;
    }
}

void launch_scale_dev_sl(const SliceMap& m, int nsl, double* x, const GmState* st, int j, cudaStream_t s) {
    launch_pdl(k_scal_dev_sl, dim3(kry_blocks(m.nl >> 1), nsl), dim3(KT), s, m, x, st, j);
}

void launch_scale_inv_sqrt(int n, double* x, const double* nrm2, cudaStream_t s) {
    launch_pdl(k_scal, dim3(kry_blocks((n + 1) >> 1)), dim3(KT), s, n, x, 0.0, nrm2);
}

void launch_scale(int n, double* x, double a, cudaStream_t s) {
    launch_pdl(k_scal, dim3(kry_blocks((n + 1) >> 1)), dim3(KT), s, n, x, a, nullptr);
}

template void launch_combine<double>(int, int, const double* const*, const double*, double*,
                                     cudaStream_t);
template void launch_combine<float>(int, int, const float* const*, const double*, double*,
                                    cudaStream_t);
template void launch_combine_dev<double>(int, int, const double* const*, const double*, const int*,
                                         double*, cudaStream_t);
template void launch_combine_dev<float>(int, int, const float* const*, const double*, const int*,
                                        double*, cudaStream_t);
template void launch_combine_dev_sl<double>(const SliceMap&, int, int, const double* const*,
                                            const GmState*, double*, cudaStream_t);
template void launch_combine_dev_sl<float>(const SliceMap&, int, int, const float* const*,
                                           const GmState*, double*, cudaStream_t);

}  // namespace stk
