// CUDA kernels of libstokes_gb300 (sm_103a): the staggered-grid Stokes
// operator, the App. C multigrid components and the Krylov vector kernels.
//
// Reference: Cai, Nonaka, Bell, Griffith & Donev, "Efficient
// Variable-Coefficient Finite-Volume Stokes Solvers", arXiv:1308.4605.
//   Sec. 3.1  D, G, L_mu (Eq. div_stress), face density, node/edge viscosity
//   App. C    multicolour Gauss-Seidel, restriction, prolongation, coarse
//             coefficients
//
// Conventions (see internal.cuh): packed face vectors, wall faces stored as
// zeros and never written with anything else; face i of component a lies on
// the low-a side of cell i.  Every stencil below is evaluated only on faces
// that carry an unknown, so no index ever leaves its array.
#include "stencil.cuh"

#include <cmath>

namespace stk {

namespace {

using namespace st;

constexpr int TPB = 256;
constexpr int SUBG = 4;   // faces per thread of k_sub_grad

// plain decode (coefficient set-up only)
__device__ __forceinline__ void decode(int t, const int e[3], int q[3]) {
    q[0] = t % e[0];
    int r = t / e[0];
    q[1] = r % e[1];
    q[2] = r / e[1];
}

// Block ranges: blocks [start[s], start[s+1]) serve segment s.
struct Segs {
    int start[5];
    int nseg;
};

// per: faces handled by one thread
inline Segs face_segs(const Geom& g, bool with_cells, int per = 1) {
    Segs s{};
    int b = 0;
    for (int a = 0; a < g.dim; ++a) {
        s.start[a] = b;
        b += (g.fsize[a] + TPB * per - 1) / (TPB * per);
    }
    s.nseg = g.dim;
    if (with_cells) {
        s.start[g.dim] = b;
        b += (g.ncell + TPB - 1) / TPB;
        s.nseg = g.dim + 1;
    }
    s.start[s.nseg] = b;
    return s;
}

__device__ __forceinline__ int seg_of(const Segs& s, int blk, int& local) {
    int k = 0;
    while (k + 1 < s.nseg && blk >= s.start[k + 1]) ++k;
    local = (blk - s.start[k]) * blockDim.x + threadIdx.x;
    return k;
}

// ------------------------------------------------------------------ coefficients
__global__ void k_fine_faces(Geom g, const double* __restrict__ rho, double theta,
                             double* alpha, double* beta) {
    pdl_entry();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.nvel) return;
    int a = 0;
    while (a + 1 < g.dim && t >= g.foff[a + 1]) ++a;
    int q[3];
    decode_face(g, a, t - g.foff[a], q);
    if (wall_face(g, a, q)) {
        alpha[t] = 0.0;
        beta[t] = 0.0;
        return;
    }
    int qm[3] = {q[0], q[1], q[2]};
    qm[a] = step(g, a, q[a], -1);
    double rf = 0.5 * (rho[cidx(g, q)] + rho[cidx(g, qm)]);
    alpha[t] = theta * rf;
    beta[t] = 1.0 / rf;
}

// Node (2D) / edge (3D) viscosity: mean of the in-domain cells around the
// edge, zero on free-slip walls and on edges lying on two walls.
__global__ void k_fine_edges(Geom g, int p, int a, int b, const double* __restrict__ mu,
                             double* mu_e) {
    pdl_entry();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.esize[p]) return;
    int q[3];
    decode(t, g.ee[p], q);
    double acc = 0.0;
    int cnt = 0;
    for (int da = -1; da <= 0; ++da)
        for (int db = -1; db <= 0; ++db) {
            int c[3] = {q[0], q[1], q[2]};
            c[a] += da;
            c[b] += db;
            bool ok = true;
            const int axes[2] = {a, b};
            for (int m = 0; m < 2; ++m) {
                const int ax = axes[m];
                if (g.per[ax]) c[ax] = wrapm(c[ax], g.n[ax]);
                else if (c[ax] < 0 || c[ax] >= g.n[ax]) ok = false;
            }
            if (ok) {
                acc += mu[cidx(g, c)];
                ++cnt;
            }
        }
    double v = cnt ? acc / cnt : 0.0;
    bool wa = !g.per[a] && (q[a] == 0 || q[a] == g.n[a]);
    bool wb = !g.per[b] && (q[b] == 0 || q[b] == g.n[b]);
    if (wa && wb) v = 0.0;
    if (wa && ((q[a] == 0 && g.bclo[a] == FREESLIP) || (q[a] == g.n[a] && g.bchi[a] == FREESLIP)))
        v = 0.0;
    if (wb && ((q[b] == 0 && g.bclo[b] == FREESLIP) || (q[b] == g.n[b] && g.bchi[b] == FREESLIP)))
        v = 0.0;
    mu_e[t] = v;
}

// Coarse face coefficients: mean of the overlying fine faces (App. C).
__global__ void k_coarsen_faces(Geom gf, Geom gc, const double* __restrict__ af,
                                const double* __restrict__ bf, double* ac, double* bcoef) {
    pdl_entry();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= gc.nvel) return;
    int a = 0;
    while (a + 1 < gc.dim && t >= gc.foff[a + 1]) ++a;
    int Q[3];
    decode_face(gc, a, t - gc.foff[a], Q);
    double sa = 0.0, sb = 0.0;
    int cnt = 0;
    int tb[2], nt = 0;
    for (int b = 0; b < gc.dim; ++b)
        if (b != a) tb[nt++] = b;
    for (int m = 0; m < (1 << nt); ++m) {
        int q[3] = {2 * Q[0], 2 * Q[1], gc.dim == 3 ? 2 * Q[2] : Q[2]};
        for (int k = 0; k < nt; ++k) q[tb[k]] += (m >> k) & 1;
        int f = fidx(gf, a, q);
        sa += af[f];
        sb += bf[f];
        ++cnt;
    }
    ac[t] = sa / cnt;
    bcoef[t] = sb / cnt;
}

__global__ void k_coarsen_cells(Geom gf, Geom gc, const double* __restrict__ mf, double* mc) {
    pdl_entry();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= gc.ncell) return;
    int Q[3];
    decode_cell(gc, t, Q);
    double s = 0.0;
    int nz = gc.dim == 3 ? 2 : 1;
    for (int dz = 0; dz < nz; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                int q[3] = {2 * Q[0] + dx, 2 * Q[1] + dy, (gc.dim == 3 ? 2 * Q[2] : Q[2]) + dz};
                s += mf[cidx(gf, q)];
            }
    mc[t] = s / (gc.dim == 3 ? 8.0 : 4.0);
}

// Coarse node viscosity by injection (2D); coarse edge viscosity as the mean
// of the two overlying fine edges (3D), App. C.
__global__ void k_coarsen_edges(Geom gf, Geom gc, int p, int c, const double* __restrict__ ef,
                                double* ec) {
    pdl_entry();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= gc.esize[p]) return;
    int Q[3];
    decode(t, gc.ee[p], Q);
    if (gc.dim == 2) {
        int q[3] = {2 * Q[0], 2 * Q[1], Q[2]};
        ec[t] = ef[eidx(gf, p, q)];
    } else {
        int q[3] = {2 * Q[0], 2 * Q[1], 2 * Q[2]};
        double v = ef[eidx(gf, p, q)];
        q[c] += 1;
        v += ef[eidx(gf, p, q)];
        ec[t] = 0.5 * v;
    }
}

template <int DIM, bool BULK>
__global__ void k_inverse_diagonals(Geom g, Coef<double> C, Segs sg) {
    pdl_entry();
    int t;
    int s = seg_of(sg, blockIdx.x, t);
    int q[3];
    if (s == DIM) {
        if (t >= g.ncell) return;
        decode_cell(g, t, q);
        double d;
        double dummy = 0.0;
        (void)dummy;
        poisson_cell<DIM, double, double>(g, C, q, C.beta, d);   // phi unused for diag
        C.invd_p[t] = d != 0.0 ? 1.0 / d : 0.0;
        return;
    }
    if (t >= g.fsize[s]) return;
    decode_face(g, s, t, q);
    int f = g.foff[s] + t;
    if (wall_face(g, s, q)) {
        C.invd_u[f] = 0.0;
        if (C.diag_u) C.diag_u[f] = 0.0;
        return;
    }
    double dsum = 0.0;
    visc_offdiag_any<DIM, double, double, true, BULK>(s, g, C, q, C.alpha, dsum);   // N unused
    double d = C.alpha[f] + g.ih2 * dsum;
    C.invd_u[f] = d != 0.0 ? 1.0 / d : 0.0;
    if (C.diag_u) C.diag_u[f] = d;
}

// 2 mu at cells (the coefficient arrays hold the doubled viscosity)
__global__ void k_twice(int n, const double* __restrict__ mu, double* __restrict__ mu2) {
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) mu2[t] = 2.0 * mu[t];
}

// bulk term of the stress at cells: lam = gamma - 2/3 mu (Sec. 2)
__global__ void k_bulk_lambda(int n, const double* __restrict__ gamma, const double* __restrict__ mu,
                              double* __restrict__ lam) {
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) lam[t] = fma(-2.0 / 3.0, mu[t], gamma[t]);
}

// b = a converted: FP32 -> FP64 by widen() (integer instructions, exact),
// FP64 -> FP32 by the rounding conversion
template <typename TB, typename TA>
__device__ __forceinline__ TB conv(TA v) {
    if constexpr (sizeof(TB) == 8 && sizeof(TA) == 4) return widen(v);
    else return TB(v);
}

template <typename TA, typename TB>
__global__ void k_convert(int n, const TA* __restrict__ a, TB* __restrict__ b) {
    pdl_entry();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) b[t] = conv<TB>(a[t]);
}

// 16-byte loads and stores of four consecutive elements (both arrays 16-byte
// aligned): a streaming copy with one element per thread is latency-bound
// well below HBM bandwidth; four per thread, in wide accesses, keep more
// bytes in flight.
__device__ __forceinline__ void ld4(const float* p, float v[4]) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w;
}
__device__ __forceinline__ void ld4(const double* p, double v[4]) {
    const double2 x = reinterpret_cast<const double2*>(p)[0];
    const double2 y = reinterpret_cast<const double2*>(p)[1];
    v[0] = x.x, v[1] = x.y, v[2] = y.x, v[3] = y.y;
}
__device__ __forceinline__ void st4(float* p, const float v[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double v[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
template <typename TA, typename TB>
__global__ void k_convert4(int n, const TA* __restrict__ a, TB* __restrict__ b) {
    pdl_entry();
    const long long i = 4LL * (blockIdx.x * (long long)blockDim.x + threadIdx.x);
    if (i + 3 < n) {
        TA v[4];
        TB w[4];
        ld4(a + i, v);
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = conv<TB>(v[k]);
        st4(b + i, w);
    } else {
        for (long long k = i; k < n; ++k) b[k] = conv<TB>(a[k]);
    }
}

// ------------------------------------------------------------------- multigrid
// One colour of the staggered Gauss-Seidel smoother (App. C): every A-face
// with (i + j + k) % 2 == parity gets phi += D^{-1} (rhs - A phi).
// ZM: components known to be zero (first sweep from a zero initial guess).
template <int DIM, int A, typename T, bool BULK, int ZM = 0>
__global__ void __launch_bounds__(512) k_vel_gs(Geom g, Coef<T> C, int parity, T* __restrict__ phi,
                                                const T* __restrict__ rhs, int nthreads) {
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nthreads) return;
    int q[3];
    if (!decode_face_colour(g, A, parity, t, q) || wall_face(g, A, q)) return;
    vel_gs_point<DIM, A, T, BULK, ZM>(g, C, q, phi, rhs);
}

// Residual rhs - A phi.  zl >= 0: the sweeps just ended with the black
// faces of component zl, whose equations they solved exactly with every
// neighbour final, so their residual is zero (up to rounding) and is set so.
template <int DIM, typename T, bool BULK>
__global__ void __launch_bounds__(TPB) k_vel_residual(Geom g, Coef<T> C, Segs sg,
                                                      const T* __restrict__ phi,
                                                      const T* __restrict__ rhs, T* __restrict__ res,
                                                      int zl) {
    pdl_entry();
    int t;
    const int s = seg_of(sg, blockIdx.x, t);
    if (t >= g.fsize[s]) return;
    int q[3];
    decode_face(g, s, t, q);
    const int f = g.foff[s] + t;
    if (wall_face(g, s, q) || (s == zl && (csum<DIM>(q) & 1))) {
        res[f] = T(0);
        return;
    }
    res[f] = vel_res_point<DIM, T, BULK>(s, g, C, q, phi, rhs);
}

template <int DIM, typename T>
__global__ void __launch_bounds__(TPB) k_vel_restrict(Geom gf, Geom gc, Segs sg,
                                                      const T* __restrict__ res, T* __restrict__ rc) {
    pdl_entry();
    int t;
    const int a = seg_of(sg, blockIdx.x, t);
    if (t >= gc.fsize[a]) return;
    int Q[3];
    decode_face(gc, a, t, Q);
    const int f = gc.foff[a] + t;
    T v = T(0);
    if (!wall_face(gc, a, Q)) {
        if (a == 0) v = vel_restrict_point<DIM, 0, T>(gf, Q, res);
        else if (a == 1) v = vel_restrict_point<DIM, 1, T>(gf, Q, res);
        else v = vel_restrict_point<DIM, DIM == 3 ? 2 : 1, T>(gf, Q, res);
    }
    rc[f] = v;
}

template <int DIM, typename T>
__global__ void __launch_bounds__(TPB) k_vel_prolong_add(Geom gc, Geom gf, Segs sg,
                                                         const T* __restrict__ pc,
                                                         T* __restrict__ pf) {
    pdl_entry();
    int t;
    const int a = seg_of(sg, blockIdx.x, t);
    if (t >= gf.fsize[a]) return;
    int q[3];
    decode_face(gf, a, t, q);
    if (wall_face(gf, a, q)) return;
    T v;
    if (a == 0) v = vel_prolong_point<DIM, 0, T>(gc, q, pc);
    else if (a == 1) v = vel_prolong_point<DIM, 1, T>(gc, q, pc);
    else v = vel_prolong_point<DIM, DIM == 3 ? 2 : 1, T>(gc, q, pc);
    pf[gf.foff[a] + t] += v;
}

// Red-black Gauss-Seidel colour for L_rho phi = rhs (App. C).
// Z: every neighbour is zero (first colour of a sweep from a zero initial guess).
template <int DIM, typename T, bool Z = false>
__global__ void __launch_bounds__(512) k_cell_gs(Geom g, Coef<T> C, int parity, T* __restrict__ phi,
                                                 const T* __restrict__ rhs, int nthreads) {
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nthreads) return;
    int q[3];
    decode_cell_colour(g, parity, t, q);
    cell_gs_point<DIM, T, Z>(g, C, q, phi, rhs);
}

// Residual rhs - L_rho phi; zb: the sweeps just ended with the black cells,
// whose residual is then zero (see k_vel_residual).
template <int DIM, typename T>
__global__ void __launch_bounds__(TPB) k_cell_residual(Geom g, Coef<T> C, const T* __restrict__ phi,
                                                       const T* __restrict__ rhs, T* __restrict__ res,
                                                       int zb) {
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ncell) return;
    int q[3];
    decode_cell(g, t, q);
    res[t] = (zb && (csum<DIM>(q) & 1)) ? T(0) : cell_res_point<DIM, T>(g, C, q, phi, rhs);
}

template <int DIM, typename T>
__global__ void __launch_bounds__(TPB) k_cell_restrict(Geom gf, Geom gc, const T* __restrict__ res,
                                                       T* __restrict__ rc) {
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= gc.ncell) return;
    int Q[3];
    decode_cell(gc, t, Q);
    rc[t] = cell_restrict_point<DIM, T>(gf, Q, res);
}

template <int DIM, typename T>
__global__ void __launch_bounds__(TPB) k_cell_prolong_add(Geom gc, Geom gf, const T* __restrict__ pc,
                                                          T* __restrict__ pf) {
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= gf.ncell) return;
    int q[3];
    decode_cell(gf, t, q);
    int Q[3] = {q[0] >> 1, q[1] >> 1, DIM == 3 ? q[2] >> 1 : q[2]};
    pf[t] += pc[cidx(gc, Q)];
}

// -------------------------------------------------------- preconditioner algebra
template <int DIM, typename T>
__global__ void k_div_plus(Geom g, const T* __restrict__ u, const T* __restrict__ bp,
                           T* __restrict__ bc) {
    pdl_entry();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ncell) return;
    int q[3];
    decode_cell(g, t, q);
    T div = T(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int qh[3] = {q[0], q[1], q[2]};
        qh[a] = step(g, a, q[a], 1);
        div += (u[fidx(g, a, qh)] - u[fidx(g, a, q)]) * gih<T>(g);
    }
    bc[t] = div + (bp ? bp[t] : T(0));
}

template <int DIM, typename T>
__global__ void k_sub_grad(Geom g, Segs sg, const T* __restrict__ beta, const T* __restrict__ u,
                           const T* __restrict__ p, T* __restrict__ out) {
    pdl_entry();
    // SUBG consecutive faces of one component per thread, all loads before
    // the stores (more bytes in flight than one face per thread)
    int t;
    const int a = seg_of(sg, blockIdx.x, t);
    T v[SUBG];
    int f[SUBG];
#pragma unroll
    for (int k = 0; k < SUBG; ++k) {
        const int tk = t * SUBG + k;
        f[k] = -1;
        v[k] = T(0);
        if (tk >= g.fsize[a]) continue;
        int q[3];
        decode_face(g, a, tk, q);
        f[k] = g.foff[a] + tk;
        if (wall_face(g, a, q)) continue;
        int qm[3] = {q[0], q[1], q[2]};
        qm[a] = step(g, a, q[a], -1);
        const T grad = (p[cidx(g, q)] - p[cidx(g, qm)]) * gih<T>(g);
        v[k] = u[f[k]] - (beta ? beta[f[k]] : T(1)) * grad;
    }
#pragma unroll
    for (int k = 0; k < SUBG; ++k)
        if (f[k] >= 0) out[f[k]] = v[k];
}

template <int DIM, typename T, bool BULK>
__global__ void k_vel_correction_rhs(Geom g, Coef<T> C, Segs sg, const T* __restrict__ b,
                                     const T* __restrict__ p, const T* __restrict__ u,
                                     T* __restrict__ out) {
    pdl_entry();
    int t;
    int s = seg_of(sg, blockIdx.x, t);
    if (t >= g.fsize[s]) return;
    int q[3];
    decode_face(g, s, t, q);
    int f = g.foff[s] + t;
    if (wall_face(g, s, q)) {
        out[f] = T(0);
        return;
    }
    int qm[3] = {q[0], q[1], q[2]};
    qm[s] = step(g, s, q[s], -1);
    T grad = (p[cidx(g, q)] - p[cidx(g, qm)]) * gih<T>(g);
    out[f] = vel_res_point<DIM, T, BULK>(s, g, C, q, u, b) - grad;
}

template <typename T>
__global__ void k_schur_combine(int n, const double* __restrict__ theta, const T* __restrict__ phi,
                                const T* __restrict__ mu2, const T* __restrict__ lam,
                                const T* __restrict__ bc, T* __restrict__ xp) {
    pdl_entry();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    T k = mu2[t];                // 2 mu, or gamma + 4/3 mu = 2 mu + lam (Eq. Schur_app_bulk)
    if (lam) k += lam[t];
    T v = -k * bc[t];
    if (phi) v += T(*theta) * phi[t];
    xp[t] = v;
}

// --------------------------------------------------------- adjoint gradient
// Strain rate dv_a/dx_b + dv_b/dx_a (times h) on the (a, b) edge at position e,
// with the one-sided no-slip wall derivative (v_first - 0)/(h/2) (Sec. 3.1).
template <typename TV>
__device__ __forceinline__ double edge_rate_h(const Geom& g, int a, int b, const int e[3],
                                              const TV* v) {
    double r = 0.0;
    const int ab[2][2] = {{a, b}, {b, a}};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int c = ab[k][0], d = ab[k][1];   // d v_c / d x_d
        if (!g.per[c] && (e[c] == 0 || e[c] == g.n[c])) continue;   // v_c faces on a c-wall are 0
        int f[3] = {e[0], e[1], e[2]};
        if (!g.per[d] && e[d] == 0) {
            r += 2.0 * double(v[fidx(g, c, f)]);
        } else if (!g.per[d] && e[d] == g.n[d]) {
            f[d] = e[d] - 1;
            r -= 2.0 * double(v[fidx(g, c, f)]);
        } else {
            int fm[3] = {e[0], e[1], e[2]};
            f[d] = g.per[d] ? wrapm(e[d], g.n[d]) : e[d];
            fm[d] = step(g, d, e[d], -1);
            r += double(v[fidx(g, c, f)]) - double(v[fidx(g, c, fm)]);
        }
    }
    return r;
}

// dL/dlog(mu_c) and dL/drho_c from the forward velocity u and the adjoint
// velocity lambda: dL/dmu_c = lambda^T (dL_mu/dmu_c) u and
// dL/drho_c = -theta lambda^T (d rho_f/d rho_c) u (M is affine in mu, rho).
// With the stress form: -2 sum_a (D_a lambda)(D_a u) on the cell, and on each
// edge around it -(m_e w_e / cnt_e) gamma(lambda) gamma(u), cnt_e the number
// of in-domain cells around the edge, m_e its free-slip/corner mask, w_e = 1/2
// on a no-slip wall (the flux across the half cell) and 1 inside.
template <int DIM>
__global__ void k_gradient(Geom g, const double* __restrict__ mu, double theta,
                           const double* __restrict__ u, const double* __restrict__ lam,
                           double* __restrict__ glogmu, double* __restrict__ grho) {
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ncell) return;
    int q[3];
    decode_cell(g, t, q);
    double gm = 0.0, gr = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int qh[3] = {q[0], q[1], q[2]};
        qh[a] = step(g, a, q[a], 1);
        const int flo = fidx(g, a, q), fhi = fidx(g, a, qh);
        const double du = u[fhi] - u[flo];
        const double dl = lam[fhi] - lam[flo];
        gm -= 2.0 * dl * du * g.ih2;
        gr -= 0.5 * theta * (lam[flo] * u[flo] + lam[fhi] * u[fhi]);
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = a + 1; b < DIM; ++b) {
#pragma unroll
            for (int sa = 0; sa < 2; ++sa)
#pragma unroll
                for (int sb = 0; sb < 2; ++sb) {
                    int e[3] = {q[0], q[1], q[2]};
                    e[a] += sa;
                    e[b] += sb;
                    const bool wa = !g.per[a] && (e[a] == 0 || e[a] == g.n[a]);
                    const bool wb = !g.per[b] && (e[b] == 0 || e[b] == g.n[b]);
                    if (wa && wb) continue;                         // corner edge: unused
                    if (wa && ((e[a] == 0 ? g.bclo[a] : g.bchi[a]) == FREESLIP)) continue;
                    if (wb && ((e[b] == 0 ? g.bclo[b] : g.bchi[b]) == FREESLIP)) continue;
                    if (g.per[a]) e[a] = wrapm(e[a], g.n[a]);
                    if (g.per[b]) e[b] = wrapm(e[b], g.n[b]);
                    const double cnt = (wa || wb) ? 2.0 : 4.0;
                    const double w = (wa || wb) ? 0.5 : 1.0;
                    gm -= w / cnt * edge_rate_h(g, a, b, e, lam) * edge_rate_h(g, a, b, e, u) * g.ih2;
                }
        }
    glogmu[t] = mu[t] * gm;
    grho[t] = gr;
}

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;   // valid in thread 0
}

// The final sum of a cell-vector reduction and the mean, done by the block
// that finishes last (no launch of their own): out[0] = sum of the nb =
// gridDim.x block partials (thread t adds b = t, t + blockDim.x, ..., then
// block_sum), out[1] = out[0] / n; the count *cnt is reset for the next
// reduction on the stream (kernels on a stream never overlap: each waits at
// pdl_entry() for its predecessor to complete).
__device__ __forceinline__ void finish_sum(const double* part, int n, double* out, unsigned* cnt) {
    __shared__ unsigned s_last;
    __shared__ double sh[32];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(cnt, 1u) == gridDim.x - 1u ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(part + b);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        out[0] = s;
        out[1] = s / n;
        *cnt = 0u;
    }
}

// s + x[i] + x[i + st] + ... over i < n, added in that order; the loads of
// eight steps are issued before their adds (a thread of a reduction grid
// has tens of steps, each a dependent FP64 add)
template <typename T>
__device__ __forceinline__ double strided_sum(const T* __restrict__ x, int i, int n, int st) {
    constexpr int U = 8;
    double s = 0.0;
    for (; i < n - (U - 1) * st; i += U * st) {
        T v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = x[i + u * st];
#pragma unroll
        for (int u = 0; u < U; ++u) s += double(v[u]);
    }
    for (; i < n; i += st) s += double(x[i]);
    return s;
}

template <typename T>
__global__ void k_sum_partials(int n, const T* __restrict__ x, double* part, double* out, unsigned* cnt) {
    pdl_entry();
    __shared__ double sh[32];
    double s = strided_sum(x, blockIdx.x * blockDim.x + threadIdx.x, n, gridDim.x * blockDim.x);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
    finish_sum(part, n, out, cnt);
}

// out[k] = sum over RED_BLOCKS partials part[k * RED_BLOCKS + b], fixed order.
__global__ void k_final(int nk, const double* __restrict__ part, double* out) {
    pdl_entry();
    __shared__ double sh[32];
    for (int k = 0; k < nk; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < RED_BLOCKS; b += blockDim.x) s += part[k * RED_BLOCKS + b];
        s = block_sum(s, sh);
        if (threadIdx.x == 0) out[k] = s;
    }
}


template <typename T>
__global__ void k_sub_mean(int n, T* x, const double* __restrict__ sum) {
    pdl_entry();
    const T m = T(sum[1]);
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) x[t] -= m;
}

template <typename T>
__global__ void k_copy_sub_mean(int n, const T* __restrict__ in, T* out,
                                const double* __restrict__ sum) {
    pdl_entry();
    const T m = T(sum[1]);
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = in[t] - m;
}

// ----------------------------------------------------------- stacked batches
// nsl instances of n values each, one after another (a cell vector of a
// stacked batch).  The sum of each instance uses the partition and the
// order of k_sum_partials above (grid (nb, nsl), blockIdx.y the instance,
// one count per instance), so it is bitwise the sum the instance gets alone:
// out[y * ostride] the sum, out[y * ostride + 1] the mean.
template <typename T>
__global__ void k_sum_partials_sl(int n, const T* __restrict__ x, double* part, double* out, int ostride,
                                  unsigned* cnt) {
    pdl_entry();
    __shared__ double sh[32];
    const T* xs = x + (size_t)blockIdx.y * n;
    double s = strided_sum(xs, blockIdx.x * blockDim.x + threadIdx.x, n, gridDim.x * blockDim.x);
    s = block_sum(s, sh);
    double* p = part + (size_t)blockIdx.y * gridDim.x;
    if (threadIdx.x == 0) p[blockIdx.x] = s;
    finish_sum(p, n, out + (size_t)blockIdx.y * ostride, cnt + blockIdx.y);
}

// out = in - mean of the instance (in place when in == out); grid (.., nsl)
template <typename T>
__global__ void k_sub_mean_sl(int n, const T* in, T* out, const double* __restrict__ sum, int stride) {
    pdl_entry();
    const T m = T(sum[(size_t)blockIdx.y * stride + 1]);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t i = (size_t)blockIdx.y * n + t;
    if (t < n) out[i] = in[i] - m;
}

template <typename T>
__global__ void k_zero(int n, T* __restrict__ x) {
    pdl_entry();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) x[t] = T(0);
}

template <typename T>
__global__ void k_axpy(int n, T a, const T* __restrict__ x, T* __restrict__ y) {
    pdl_entry();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) y[t] += a * x[t];
}

// Right-hand side of a backward-Euler step on the a-faces: b = alpha u + f
// (alpha = rho_f / dt), zero on wall faces; f may be null.
__global__ void k_inertial_rhs(Geom g, int a, const double* __restrict__ alpha,
                               const double* u, const double* f, double* b) {
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.fsize[a]) return;
    int q[3];
    decode_face(g, a, t, q);
    b[t] = wall_face(g, a, q) ? 0.0 : fma(alpha[g.foff[a] + t], u[t], f ? f[t] : 0.0);
}

// Inhomogeneous boundary data: copy the wall faces of the a-component face
// array src into the packed vector dst (other entries untouched).
__global__ void k_copy_walls(Geom g, int a, const double* __restrict__ src, double* __restrict__ dst) {
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.fsize[a]) return;
    int q[3];
    decode_face(g, a, t, q);
    if (wall_face(g, a, q)) dst[g.foff[a] + t] = src[t];
}

// Tangential velocity U of a no-slip wall of axis d (side 0 low, 1 high) for
// component a != d: the one-sided wall derivative (u_first - U)/(h/2) adds
// 2 mu_e U / h^2 to L_mu at the first interior a-faces, i.e. c -= 2 mu_e U / h^2
// in the momentum rows.  U is indexed by the a-face position without axis d.
__global__ void k_wall_tangential(Geom g, const double* __restrict__ mu_e, int d, int side, int a,
                                  const double* __restrict__ U, double* c) {
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.fsize[a]) return;
    int q[3];
    decode_face(g, a, t, q);
    if (wall_face(g, a, q) || q[d] != (side ? g.n[d] - 1 : 0)) return;
    int qe[3] = {q[0], q[1], q[2]};
    if (side) qe[d] = g.n[d];
    const int p = a + d - 1;
    int c0 = -1, c1 = -1;
    for (int k = 0; k < 3; ++k)
        if (k != d) { if (c0 < 0) c0 = k; else c1 = k; }
    const int iu = q[c1] * g.fe[a][c0] + q[c0];
    c[g.foff[a] + t] -= 2.0 * mu_e[eidx(g, p, qe)] * U[iu] * g.ih2;
}

__global__ void k_check_fields(int n, const double* __restrict__ rho, const double* __restrict__ mu,
                               double* part) {
    pdl_entry();
    __shared__ double sh[32];
    double bad = 0.0, nonpos = 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        double r = rho[t], m = mu[t];
        if (!isfinite(r) || !isfinite(m)) bad += 1.0;
        else if (r <= 0.0 || m < 0.0) nonpos += 1.0;
    }
    double s = block_sum(bad, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
    s = block_sum(nonpos, sh);
    if (threadIdx.x == 0) part[RED_BLOCKS + blockIdx.x] = s;
}

inline int nblk(long long n) { return (int)((n + TPB - 1) / TPB); }

}  // namespace

// ============================================================== launch wrappers
void launch_fine_coefficients(const Geom& g, const double* rho, const double* mu, double theta,
                              Coef<double> C, cudaStream_t s) {
    launch_pdl(k_fine_faces, dim3(nblk(g.nvel)), dim3(TPB), s, g, rho, theta, C.alpha, C.beta);
    launch_pdl(k_twice, dim3(nblk(g.ncell)), dim3(TPB), s, g.ncell, mu, C.mu2_c);
    for (int a = 0; a < g.dim; ++a)
        for (int b = a + 1; b < g.dim; ++b) {
            int p = a + b - 1;
            launch_pdl(k_fine_edges, dim3(nblk(g.esize[p])), dim3(TPB), s, g, p, a, b, mu, C.mu_e[p]);
        }
}

void launch_coarsen_coefficients(const Geom& gf, Coef<double> Cf, const Geom& gc, Coef<double> Cc,
                                 cudaStream_t s) {
    launch_pdl(k_coarsen_faces, dim3(nblk(gc.nvel)), dim3(TPB), s, gf, gc, Cf.alpha, Cf.beta, Cc.alpha, Cc.beta);
    launch_pdl(k_coarsen_cells, dim3(nblk(gc.ncell)), dim3(TPB), s, gf, gc, Cf.mu2_c, Cc.mu2_c);
    if (Cf.lam_c && Cc.lam_c)   // bulk term: cell average, like mu
        launch_pdl(k_coarsen_cells, dim3(nblk(gc.ncell)), dim3(TPB), s, gf, gc, Cf.lam_c, Cc.lam_c);
    for (int a = 0; a < gc.dim; ++a)
        for (int b = a + 1; b < gc.dim; ++b) {
            int p = a + b - 1;
            int c = 3 - a - b;
            launch_pdl(k_coarsen_edges, dim3(nblk(gc.esize[p])), dim3(TPB), s, gf, gc, p, c, Cf.mu_e[p], Cc.mu_e[p]);
        }
}

void launch_bulk_lambda(int n, const double* gamma, const double* mu, double* lam, cudaStream_t s) {
    launch_pdl(k_bulk_lambda, dim3(nblk(n)), dim3(TPB), s, n, gamma, mu, lam);
}

void launch_inverse_diagonals(const Geom& g, Coef<double> C, cudaStream_t s) {
    Segs sg = face_segs(g, true);
    const bool bk = C.lam_c != nullptr;
    if (g.dim == 2) launch_pdl(bk ? k_inverse_diagonals<2, true> : k_inverse_diagonals<2, false>, dim3(sg.start[sg.nseg]), dim3(TPB), s, g, C, sg);
    else launch_pdl(bk ? k_inverse_diagonals<3, true> : k_inverse_diagonals<3, false>, dim3(sg.start[sg.nseg]), dim3(TPB), s, g, C, sg);
}

template <typename TA, typename TB>
void launch_convert(int n, const TA* a, TB* b, cudaStream_t s) {
    if (n <= 0) return;
    const bool wide = ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0;
    if (wide) launch_pdl(k_convert4<TA, TB>, dim3(nblk((n + 3) / 4)), dim3(TPB), s, n, a, b);
    else launch_pdl(k_convert<TA, TB>, dim3(nblk(n)), dim3(TPB), s, n, a, b);
}

void launch_convert_coefficients(const Geom& g, Coef<double> C, Coef<float> F, cudaStream_t s) {
    // F.diag_u stays null: the FP32 residual forms the diagonal on the fly
    launch_convert(g.nvel, C.alpha, F.alpha, s);
    launch_convert(g.nvel, C.beta, F.beta, s);
    launch_convert(g.ncell, C.mu2_c, F.mu2_c, s);
    for (int p = 0; p < 3; ++p)
        if (g.esize[p] > 0 && C.mu_e[p]) launch_convert(g.esize[p], C.mu_e[p], F.mu_e[p], s);
    launch_convert(g.nvel, C.invd_u, F.invd_u, s);
    launch_convert(g.ncell, C.invd_p, F.invd_p, s);
    if (C.lam_c && F.lam_c) launch_convert(g.ncell, C.lam_c, F.lam_c, s);
}

template <typename T>
void launch_vel_gs_colour(const Geom& g, Coef<T> C, int comp, int parity, T* phi, const T* rhs,
                          cudaStream_t s, int tpb, bool first) {
    const int nt = ((g.fe[comp][0] + 1) / 2) * g.fe[comp][1] * g.fe[comp][2];
    const int nb = (nt + tpb - 1) / tpb;
    const bool bk = C.lam_c != nullptr;
    if (first && !bk) {
        // first sweep from zero, red (parity 0) before black, components in
        // order: zero are the faces of comp not yet swept and the later components
        const int zm = (parity == 0 ? 1 << comp : 0) | (((1 << g.dim) - 1) & ~((2 << comp) - 1));
        void (*k)(Geom, Coef<T>, int, T*, const T*, int) = nullptr;
        if (g.dim == 2) {
            if (zm == 3) k = k_vel_gs<2, 0, T, false, 3>;
            else if (zm == 2) k = comp == 0 ? k_vel_gs<2, 0, T, false, 2> : k_vel_gs<2, 1, T, false, 2>;
        } else {
            if (zm == 7) k = k_vel_gs<3, 0, T, false, 7>;
            else if (zm == 6) k = comp == 0 ? k_vel_gs<3, 0, T, false, 6> : k_vel_gs<3, 1, T, false, 6>;
            else if (zm == 4) k = comp == 1 ? k_vel_gs<3, 1, T, false, 4> : k_vel_gs<3, 2, T, false, 4>;
        }
        if (k) {
            launch_pdl(k, dim3(nb), dim3(tpb), s, g, C, parity, phi, rhs, nt);
            return;
        }
    }
#define STK_VGS(D, A) (bk ? k_vel_gs<D, A, T, true> : k_vel_gs<D, A, T, false>)
    if (g.dim == 2) {
        if (comp == 0) launch_pdl(STK_VGS(2, 0), dim3(nb), dim3(tpb), s, g, C, parity, phi, rhs, nt);
        else launch_pdl(STK_VGS(2, 1), dim3(nb), dim3(tpb), s, g, C, parity, phi, rhs, nt);
    } else {
        if (comp == 0) launch_pdl(STK_VGS(3, 0), dim3(nb), dim3(tpb), s, g, C, parity, phi, rhs, nt);
        else if (comp == 1) launch_pdl(STK_VGS(3, 1), dim3(nb), dim3(tpb), s, g, C, parity, phi, rhs, nt);
        else launch_pdl(STK_VGS(3, 2), dim3(nb), dim3(tpb), s, g, C, parity, phi, rhs, nt);
    }
#undef STK_VGS
}

template <typename T>
void launch_vel_residual(const Geom& g, Coef<T> C, const T* phi, const T* rhs, T* res,
                         cudaStream_t s, bool after_sweep) {
    const int zl = after_sweep ? g.dim - 1 : -1;
    Segs sg = face_segs(g, false);
    const bool bk = C.lam_c != nullptr;
    if (g.dim == 2) launch_pdl(bk ? k_vel_residual<2, T, true> : k_vel_residual<2, T, false>, dim3(sg.start[sg.nseg]), dim3(TPB), s, g, C, sg, phi, rhs, res, zl);
    else launch_pdl(bk ? k_vel_residual<3, T, true> : k_vel_residual<3, T, false>, dim3(sg.start[sg.nseg]), dim3(TPB), s, g, C, sg, phi, rhs, res, zl);
}

template <typename T>
void launch_vel_restrict(const Geom& gf, const T* res, const Geom& gc, T* rc, cudaStream_t s) {
    Segs sg = face_segs(gc, false);
    if (gf.dim == 2) launch_pdl(k_vel_restrict<2, T>, dim3(sg.start[sg.nseg]), dim3(TPB), s, gf, gc, sg, res, rc);
    else launch_pdl(k_vel_restrict<3, T>, dim3(sg.start[sg.nseg]), dim3(TPB), s, gf, gc, sg, res, rc);
}

template <typename T>
void launch_vel_prolong_add(const Geom& gc, const T* pc, const Geom& gf, T* pf, cudaStream_t s) {
    Segs sg = face_segs(gf, false);
    if (gf.dim == 2) launch_pdl(k_vel_prolong_add<2, T>, dim3(sg.start[sg.nseg]), dim3(TPB), s, gc, gf, sg, pc, pf);
    else launch_pdl(k_vel_prolong_add<3, T>, dim3(sg.start[sg.nseg]), dim3(TPB), s, gc, gf, sg, pc, pf);
}

template <typename T>
void launch_cell_gs_colour(const Geom& g, Coef<T> C, int parity, T* phi, const T* rhs,
                           cudaStream_t s, int tpb, bool first) {
    const int nt = (g.n[0] / 2) * g.n[1] * g.n[2];
    const int nb = (nt + tpb - 1) / tpb;
    const bool z = first && parity == 0;   // red first: all its neighbours are black
    if (g.dim == 2)
        launch_pdl(z ? k_cell_gs<2, T, true> : k_cell_gs<2, T>, dim3(nb), dim3(tpb), s, g, C, parity, phi, rhs, nt);
    else
        launch_pdl(z ? k_cell_gs<3, T, true> : k_cell_gs<3, T>, dim3(nb), dim3(tpb), s, g, C, parity, phi, rhs, nt);
}

template <typename T>
void launch_cell_residual(const Geom& g, Coef<T> C, const T* phi, const T* rhs, T* res,
                          cudaStream_t s, bool after_sweep) {
    const int zb = after_sweep ? 1 : 0;
    if (g.dim == 2) launch_pdl(k_cell_residual<2, T>, dim3(nblk(g.ncell)), dim3(TPB), s, g, C, phi, rhs, res, zb);
    else launch_pdl(k_cell_residual<3, T>, dim3(nblk(g.ncell)), dim3(TPB), s, g, C, phi, rhs, res, zb);
}

template <typename T>
void launch_cell_restrict(const Geom& gf, const T* res, const Geom& gc, T* rc, cudaStream_t s) {
    if (gf.dim == 2) launch_pdl(k_cell_restrict<2, T>, dim3(nblk(gc.ncell)), dim3(TPB), s, gf, gc, res, rc);
    else launch_pdl(k_cell_restrict<3, T>, dim3(nblk(gc.ncell)), dim3(TPB), s, gf, gc, res, rc);
}

template <typename T>
void launch_cell_prolong_add(const Geom& gc, const T* pc, const Geom& gf, T* pf, cudaStream_t s) {
    if (gf.dim == 2) launch_pdl(k_cell_prolong_add<2, T>, dim3(nblk(gf.ncell)), dim3(TPB), s, gc, gf, pc, pf);
    else launch_pdl(k_cell_prolong_add<3, T>, dim3(nblk(gf.ncell)), dim3(TPB), s, gc, gf, pc, pf);
}

template <typename T>
void launch_div_plus(const Geom& g, const T* u, const T* bp, T* bc, cudaStream_t s) {
    if (g.dim == 2) launch_pdl(k_div_plus<2, T>, dim3(nblk(g.ncell)), dim3(TPB), s, g, u, bp, bc);
    else launch_pdl(k_div_plus<3, T>, dim3(nblk(g.ncell)), dim3(TPB), s, g, u, bp, bc);
}

template <typename T>
void launch_sub_grad(const Geom& g, const T* beta, const T* u, const T* p, T* out, cudaStream_t s) {
    Segs sg = face_segs(g, false, SUBG);
    if (g.dim == 2) launch_pdl(k_sub_grad<2, T>, dim3(sg.start[sg.nseg]), dim3(TPB), s, g, sg, beta, u, p, out);
    else launch_pdl(k_sub_grad<3, T>, dim3(sg.start[sg.nseg]), dim3(TPB), s, g, sg, beta, u, p, out);
}

template <typename T>
void launch_vel_correction_rhs(const Geom& g, Coef<T> C, const T* b, const T* p, const T* u,
                               T* out, cudaStream_t s) {
    Segs sg = face_segs(g, false);
    if (g.dim == 2)
        launch_pdl(C.lam_c ? k_vel_correction_rhs<2, T, true> : k_vel_correction_rhs<2, T, false>, dim3(sg.start[sg.nseg]), dim3(TPB), s, g, C, sg, b, p, u, out);
    else
        launch_pdl(C.lam_c ? k_vel_correction_rhs<3, T, true> : k_vel_correction_rhs<3, T, false>, dim3(sg.start[sg.nseg]), dim3(TPB), s, g, C, sg, b, p, u, out);
}

template <typename T>
void launch_schur_combine(int n, const double* theta, const T* phi, const T* mu2, const T* lam,
                          const T* bc, T* xp, cudaStream_t s) {
    launch_pdl(k_schur_combine<T>, dim3(nblk(n)), dim3(TPB), s, n, theta, phi, mu2, lam, bc, xp);
}

// blocks of a cell-vector sum: one value per thread at least, at most RED_BLOCKS
inline int sum_blocks(int n) {
    const int b = (n + RED_THREADS - 1) / RED_THREADS;
    return b < 1 ? 1 : (b > RED_BLOCKS ? RED_BLOCKS : b);
}

template <typename T>
void launch_sum(int n, const T* x, double* scratch, double* out, unsigned* cnt, cudaStream_t s) {
    launch_pdl(k_sum_partials<T>, dim3(sum_blocks(n)), dim3(RED_THREADS), s, n, x, scratch, out, cnt);
}

template <typename T>
void launch_sub_mean(int n, T* x, const double* sum, cudaStream_t s) {
    launch_pdl(k_sub_mean<T>, dim3(nblk(n)), dim3(TPB), s, n, x, sum);
}

template <typename T>
void launch_copy_sub_mean(int n, const T* in, T* out, const double* sum, cudaStream_t s) {
    launch_pdl(k_copy_sub_mean<T>, dim3(nblk(n)), dim3(TPB), s, n, in, out, sum);
}

template <typename T>
void launch_sum_sl(int n, int nsl, const T* x, double* scratch, double* out, int ostride, unsigned* cnt,
                   cudaStream_t s) {
    launch_pdl(k_sum_partials_sl<T>, dim3(sum_blocks(n), nsl), dim3(RED_THREADS), s, n, x, scratch, out,
               ostride, cnt);
}

template <typename T>
void launch_sub_mean_sl(int n, int nsl, const T* in, T* out, const double* sum, int stride, cudaStream_t s) {
    launch_pdl(k_sub_mean_sl<T>, dim3(nblk(n), nsl), dim3(TPB), s, n, in, out, sum, stride);
}

template <typename T>
void launch_zero(int n, T* x, cudaStream_t s) {
    const int nb = nblk(n) < 1216 ? nblk(n) : 1216;
    launch_pdl(k_zero<T>, dim3(nb > 0 ? nb : 1), dim3(TPB), s, n, x);
}

template <typename T>
void launch_axpy(int n, T a, const T* x, T* y, cudaStream_t s) {
    launch_pdl(k_axpy<T>, dim3(nblk(n)), dim3(TPB), s, n, a, x, y);
}

void launch_inertial_rhs(const Geom& g, int a, const double* alpha, const double* u,
                         const double* f, double* b, cudaStream_t s) {
    launch_pdl(k_inertial_rhs, dim3(nblk(g.fsize[a])), dim3(TPB), s, g, a, alpha, u, f, b);
}

void launch_copy_walls(const Geom& g, int a, const double* src, double* dst, cudaStream_t s) {
    launch_pdl(k_copy_walls, dim3(nblk(g.fsize[a])), dim3(TPB), s, g, a, src, dst);
}

void launch_wall_tangential(const Geom& g, const double* mu_e, int d, int side, int a,
                            const double* U, double* c, cudaStream_t s) {
    launch_pdl(k_wall_tangential, dim3(nblk(g.fsize[a])), dim3(TPB), s, g, mu_e, d, side, a, U, c);
}

void launch_gradient(const Geom& g, const double* mu, double theta, const double* u,
                     const double* lam, double* glogmu, double* grho, cudaStream_t s) {
    if (g.dim == 2) launch_pdl(k_gradient<2>, dim3(nblk(g.ncell)), dim3(TPB), s, g, mu, theta, u, lam, glogmu, grho);
    else launch_pdl(k_gradient<3>, dim3(nblk(g.ncell)), dim3(TPB), s, g, mu, theta, u, lam, glogmu, grho);
}

void launch_check_fields(int n, const double* rho, const double* mu, double* scratch, double* out,
                         cudaStream_t s) {
    launch_pdl(k_check_fields, dim3(RED_BLOCKS), dim3(RED_THREADS), s, n, rho, mu, scratch);
    launch_pdl(k_final, dim3(1), dim3(RED_THREADS), s, 2, scratch, out);
}

// explicit instantiations
#define STK_INST(T)                                                                                \
    template void launch_vel_gs_colour<T>(const Geom&, Coef<T>, int, int, T*, const T*,          \
                                          cudaStream_t, int, bool);                                \
    template void launch_vel_residual<T>(const Geom&, Coef<T>, const T*, const T*, T*,           \
                                         cudaStream_t, bool);                                      \
    template void launch_vel_restrict<T>(const Geom&, const T*, const Geom&, T*, cudaStream_t);  \
    template void launch_vel_prolong_add<T>(const Geom&, const T*, const Geom&, T*,              \
                                            cudaStream_t);                                         \
    template void launch_cell_gs_colour<T>(const Geom&, Coef<T>, int, T*, const T*,              \
                                           cudaStream_t, int, bool);                               \
    template void launch_cell_residual<T>(const Geom&, Coef<T>, const T*, const T*, T*,          \
                                          cudaStream_t, bool);                                     \
    template void launch_cell_restrict<T>(const Geom&, const T*, const Geom&, T*, cudaStream_t); \
    template void launch_cell_prolong_add<T>(const Geom&, const T*, const Geom&, T*,             \
                                             cudaStream_t);                                        \
    template void launch_div_plus<T>(const Geom&, const T*, const T*, T*, cudaStream_t);         \
    template void launch_sub_grad<T>(const Geom&, const T*, const T*, const T*, T*,              \
                                     cudaStream_t);                                                \
    template void launch_vel_correction_rhs<T>(const Geom&, Coef<T>, const T*, const T*,         \
                                               const T*, T*, cudaStream_t);                        \
    template void launch_schur_combine<T>(int, const double*, const T*, const T*, const T*,      \
                                          const T*, T*,                                            \
                                          cudaStream_t);                                           \
    template void launch_sum<T>(int, const T*, double*, double*, unsigned*, cudaStream_t);       \
    template void launch_sum_sl<T>(int, int, const T*, double*, double*, int, unsigned*,         \
                                   cudaStream_t);                                                  \
    template void launch_sub_mean_sl<T>(int, int, const T*, T*, const double*, int, cudaStream_t); \
    template void launch_sub_mean<T>(int, T*, const double*, cudaStream_t);                      \
    template void launch_copy_sub_mean<T>(int, const T*, T*, const double*, cudaStream_t);       \
    template void launch_axpy<T>(int, T, const T*, T*, cudaStream_t);                            \
    template void launch_zero<T>(int, T*, cudaStream_t);
STK_INST(double)
STK_INST(float)
#undef STK_INST
template void launch_convert<double, float>(int, const double*, float*, cudaStream_t);
template void launch_convert<float, double>(int, const float*, double*, cudaStream_t);

#ifdef STK_BOUNDS_CHECK
namespace {
// index n against length n: recorded as out of range; no memory is accessed
__global__ void k_oob_selftest(int n) {
    if (threadIdx.x == 0 && blockIdx.x == 0) (void)STK_IDX(n, n, 2);
}
}  // namespace
void launch_oob_selftest(int n, cudaStream_t s) { k_oob_selftest<<<1, 32, 0, s>>>(n); }
#endif
STK_OOB_READER(kernels)

}  // namespace stk
