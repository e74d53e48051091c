// Device-side stencils of the staggered Stokes operator and of the App. C
// multigrid, as per-point functions shared by the grid-wide kernels
// (kernels.cu) and the single-block coarse-level kernel (coarse.cu).
//
// Reference: Cai, Nonaka, Bell, Griffith & Donev, arXiv:1308.4605,
// Sec. 3.1 (Eq. div_stress, wall closures) and App. C (multicolour
// Gauss-Seidel, restriction, prolongation).
//
// Conventions: packed face vectors (components x, y[, z], x fastest), wall
// faces stored as zeros and never written; face i of component a lies on the
// low-a side of cell i.  Every stencil is evaluated only on faces that carry
// an unknown, so no index leaves its array.  Arrays that a V-cycle writes
// (phi, rhs, residuals) are read with ordinary coherent loads, never through
// the read-only path: the coarse-level kernel reads them again after a
// __syncthreads() within the same launch.  Only coefficients use __ldg.
// Every product that is added to something is written as an explicit fma,
// so that the compiler's contraction choices cannot differ between the
// kernels that inline these functions: the per-colour, two-colour and
// coarse-level kernels then give bitwise the same results.
#pragma once
#include "internal.cuh"

namespace stk {
namespace st {

__host__ __device__ __forceinline__ int wrapm(int i, int n) {
    return i < 0 ? i + n : (i >= n ? i - n : i);
}
__device__ __forceinline__ int fidx(const Geom& g, int a, const int q[3]) {
    return STK_IDX(g.foff[a] + (q[2] * g.fe[a][1] + q[1]) * g.fe[a][0] + q[0], g.nvel, 1);
}
__device__ __forceinline__ int cidx(const Geom& g, const int q[3]) {
    return STK_IDX((q[2] * g.n[1] + q[1]) * g.n[0] + q[0], g.ncell, 2);
}
__device__ __forceinline__ int eidx(const Geom& g, int p, const int q[3]) {
    return STK_IDX((q[2] * g.ee[p][1] + q[1]) * g.ee[p][0] + q[0], g.esize[p], 3);
}
// t -> (i, j, k) over the face array of component a
__device__ __forceinline__ void decode_face(const Geom& g, int a, int t, int q[3]) {
    const int r = fdiv(t, g.fd_e0[a]);
    q[0] = t - r * g.fe[a][0];
    q[2] = fdiv(r, g.fd_e1[a]);
    q[1] = r - q[2] * g.fe[a][1];
}
__device__ __forceinline__ void decode_cell(const Geom& g, int t, int q[3]) {
    const int r = fdiv(t, g.fd_n0);
    q[0] = t - r * g.n[0];
    q[2] = fdiv(r, g.fd_n1);
    q[1] = r - q[2] * g.n[1];
}
// The colour index i + j (+ k in 3D).  In 2D the third index numbers the
// instances of a stacked batch and takes no part in the colouring, so each
// instance is swept exactly as it would be alone.
__device__ __forceinline__ int csum(const Geom& g, const int q[3]) {
    return q[0] + q[1] + (g.dim == 3 ? q[2] : 0);
}
template <int DIM>
__device__ __forceinline__ int csum(const int q[3]) {
    return q[0] + q[1] + (DIM == 3 ? q[2] : 0);
}
// t-th face of component a with csum % 2 == parity; false past the end
__device__ __forceinline__ bool decode_face_colour(const Geom& g, int a, int parity, int t, int q[3]) {
    const int half = (g.fe[a][0] + 1) >> 1;
    const int r = fdiv(t, g.fd_h0[a]);
    const int xh = t - r * half;
    q[2] = fdiv(r, g.fd_e1[a]);
    q[1] = r - q[2] * g.fe[a][1];
    q[0] = 2 * xh + ((q[1] + (g.dim == 3 ? q[2] : 0) + parity) & 1);
    return q[0] < g.fe[a][0];
}
__device__ __forceinline__ void decode_cell_colour(const Geom& g, int parity, int t, int q[3]) {
    const int half = g.n[0] >> 1;
    const int r = fdiv(t, g.fd_nh0);
    const int xh = t - r * half;
    q[2] = fdiv(r, g.fd_n1);
    q[1] = r - q[2] * g.n[1];
    q[0] = 2 * xh + ((q[1] + (g.dim == 3 ? q[2] : 0) + parity) & 1);
}
__device__ __forceinline__ bool wall_face(const Geom& g, int a, const int q[3]) {
    return !g.per[a] && (q[a] == 0 || q[a] == g.n[a]);
}
__device__ __forceinline__ int step(const Geom& g, int ax, int i, int d) {
    return g.per[ax] ? wrapm(i + d, g.n[ax]) : i + d;
}
template <typename T> __device__ __forceinline__ T ld(const T* p) { return __ldg(p); }


template <typename T> __device__ __forceinline__ T gih(const Geom& g);
template <> __device__ __forceinline__ double gih<double>(const Geom& g) { return g.ih; }
template <> __device__ __forceinline__ float gih<float>(const Geom& g) { return g.ihf; }
template <typename T> __device__ __forceinline__ T gih2(const Geom& g);
template <> __device__ __forceinline__ double gih2<double>(const Geom& g) { return g.ih2; }
template <> __device__ __forceinline__ float gih2<float>(const Geom& g) { return g.ih2f; }

// the axes other than A (compile time)
template <int DIM, int A> struct Trans;
template <int A> struct Trans<2, A> { static constexpr int n = 1, b0 = 1 - A, b1 = 1 - A; };
template <int A> struct Trans<3, A> {
    static constexpr int n = 2, b0 = (A + 1) % 3, b1 = (A + 2) % 3;
};

// h^2 (L_mu phi)_A at the interior A-face q (Eq. div_stress with the wall
// closures of Sec. 3.1), grid scaling factored out, arithmetic in T, split
// into its off-diagonal part: h^2 L_A = N - phi_A dsum,
//   N    = 2 (mu_hi phi_A[+a] + mu_lo phi_A[-a])
//          + sum_B mu_e,hi (phi_A[+b] + dphi_B/dx_A|hi) + mu_e,lo (phi_A[-b] - dphi_B/dx_A|lo)
//   dsum = 2 (mu_hi + mu_lo) + sum_B (f_hi mu_e,hi + f_lo mu_e,lo),
// with phi_A beyond a wall omitted from N (f = 2 there: the one-sided
// derivative over h/2, Sec. 3.1; f = 1 inside).  A Gauss-Seidel step is then
// phi_A <- (rhs + N / h^2) / (alpha + dsum / h^2) with no term in the old
// phi_A, and the operator is A phi = diag phi_A - N / h^2.
// With bulk viscosity (Sec. 2: + (gamma - 2/3 mu)(div u) I in the stress,
// lam = gamma - 2/3 mu at cells) the normal stresses of the two cells gain
// lam times their divergence: N += lam_hi (phi_A[+a] + sum_B dphi_B|hi)
// + lam_lo (phi_A[-a] - sum_B dphi_B|lo), dphi_B the B-face difference
// across the cell, and dsum += lam_hi + lam_lo.
// Where the stencil of the A-face q reads its values: indices of phi_A at
// q +- e_A and at q +- e_B, of mu at the cells q and q - e_A, of mu_e on the
// edges q and q + e_B, and of phi_B at the B-faces q, q - e_A, q + e_B and
// q + e_B - e_A, for the transverse axes B in increasing order (slot j).
// wlo / whi: q is next to a wall of axis B on the low / high side.
struct Nbr {
    int a_p, a_m, c_h, c_l;
    int e_lo[2], e_hi[2], b_q[2], b_r0[2], b_qe[2], b_r2[2], a_bp[2], a_bm[2];
    bool wlo[2], whi[2];
};

// transverse axis of slot j (increasing order)
__host__ __device__ constexpr int trans_axis(int dim, int a, int j) {
    return dim == 2 ? 1 - a : (j == 0 ? (a == 0 ? 1 : 0) : (a == 2 ? 1 : 2));
}

// Index table from linear strides: one base index per array and constant
// offsets, with a branch-free correction on the faces next to a periodic
// seam (equal to the coordinate form, whose stepping wraps there).
template <int DIM, int A>
__device__ __forceinline__ void nbr_lin(const Geom& g, const int q[3], Nbr& X) {
    int kp[3], km[3];   // +1 / -1 steps in units of the stride: 1, or 1 - n across a seam
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        kp[d] = (g.per[d] && q[d] == g.n[d] - 1) ? 1 - g.n[d] : 1;
        km[d] = (g.per[d] && q[d] == 0) ? 1 - g.n[d] : 1;
    }
    const int sA[3] = {1, g.fe[A][0], g.fe[A][0] * g.fe[A][1]};
    const int f = fidx(g, A, q);
    X.a_p = f + kp[A] * sA[A];
    X.a_m = f - km[A] * sA[A];
    const int sc[3] = {1, g.n[0], g.n[0] * g.n[1]};
    X.c_h = cidx(g, q);
    X.c_l = X.c_h - km[A] * sc[A];
#pragma unroll
    for (int j = 0; j < DIM - 1; ++j) {
        const int B = trans_axis(DIM, A, j);
        const int P = A + B - 1;
        const int se[3] = {1, g.ee[P][0], g.ee[P][0] * g.ee[P][1]};
        const int e = eidx(g, P, q);
        X.e_lo[j] = e;
        X.e_hi[j] = e + kp[B] * se[B];
        const int sB[3] = {1, g.fe[B][0], g.fe[B][0] * g.fe[B][1]};
        const int fb = fidx(g, B, q);
        X.b_q[j] = fb;
        X.b_r0[j] = fb - km[A] * sB[A];
        X.b_qe[j] = fb + kp[B] * sB[B];
        X.b_r2[j] = X.b_qe[j] - km[A] * sB[A];
        X.a_bp[j] = f + kp[B] * sA[B];
        X.a_bm[j] = f - km[B] * sA[B];
        X.wlo[j] = !g.per[B] && q[B] == 0;
        X.whi[j] = !g.per[B] && q[B] == g.n[B] - 1;
#ifdef STK_BOUNDS_CHECK
        X.e_lo[j] = STK_IDX(X.e_lo[j], g.esize[P], 3);
        X.e_hi[j] = STK_IDX(X.e_hi[j], g.esize[P], 3);
        X.b_q[j] = STK_IDX(X.b_q[j], g.nvel, 1);
        X.b_r0[j] = STK_IDX(X.b_r0[j], g.nvel, 1);
        X.b_qe[j] = STK_IDX(X.b_qe[j], g.nvel, 1);
        X.b_r2[j] = STK_IDX(X.b_r2[j], g.nvel, 1);
        if (!X.whi[j]) X.a_bp[j] = STK_IDX(X.a_bp[j], g.nvel, 1);
        if (!X.wlo[j]) X.a_bm[j] = STK_IDX(X.a_bm[j], g.nvel, 1);
#endif
    }
#ifdef STK_BOUNDS_CHECK
    X.a_p = STK_IDX(X.a_p, g.nvel, 1);
    X.a_m = STK_IDX(X.a_m, g.nvel, 1);
    X.c_h = STK_IDX(X.c_h, g.ncell, 2);
    X.c_l = STK_IDX(X.c_l, g.ncell, 2);
#endif
}

// Index table from coordinates; aidx(r) gives the index of phi_A at the
// A-face r (a global index, or a shared-memory slot), B-faces are global.
template <int DIM, int A, typename AI>
__device__ __forceinline__ void nbr_coord(const Geom& g, const int q[3], const AI& aidx, Nbr& X) {
    int qp[3] = {q[0], q[1], q[2]};
    int qm[3] = {q[0], q[1], q[2]};
    qp[A] = step(g, A, q[A], 1);
    qm[A] = step(g, A, q[A], -1);
    X.a_p = aidx(qp);
    X.a_m = aidx(qm);
    X.c_h = cidx(g, q);
    X.c_l = cidx(g, qm);
#pragma unroll
    for (int j = 0; j < DIM - 1; ++j) {
        const int B = trans_axis(DIM, A, j);
        const int P = A + B - 1;
        int qe[3] = {q[0], q[1], q[2]};
        qe[B] = step(g, B, q[B], 1);
        X.e_lo[j] = eidx(g, P, q);
        X.e_hi[j] = eidx(g, P, qe);
        int r0[3] = {q[0], q[1], q[2]};
        r0[A] = qm[A];
        int r2[3] = {qe[0], qe[1], qe[2]};
        r2[A] = qm[A];
        X.b_q[j] = fidx(g, B, q);
        X.b_r0[j] = fidx(g, B, r0);
        X.b_qe[j] = fidx(g, B, qe);
        X.b_r2[j] = fidx(g, B, r2);
        X.wlo[j] = !g.per[B] && q[B] == 0;
        X.whi[j] = !g.per[B] && q[B] == g.n[B] - 1;
        X.a_bp[j] = X.whi[j] ? 0 : aidx(qe);
        int qb[3] = {q[0], q[1], q[2]};
        qb[B] = step(g, B, q[B], -1);
        X.a_bm[j] = X.wlo[j] ? 0 : aidx(qb);
    }
}

// The arithmetic: ga(i) reads phi_A at index i, gb(B, i) phi_B at index i.
// ZM: components known to be zero (bit c for phi_c), as in the first sweep
// from a zero initial guess, where the faces of the colour not yet updated
// and the components after A are still zero.  Their terms are left out
// rather than multiplied by zero: the same sum up to the sign of a zero.
template <int DIM, int A, typename T, bool DIAG, bool BULK, int ZM = 0, typename GA, typename GB>
__device__ __forceinline__ T visc_offdiag_tab(const Coef<T>& C, const Nbr& X, const GA& ga,
                                              const GB& gb, T& dsum) {
    constexpr bool za = (ZM >> A) & 1;
    T N = T(0);
    T mh = T(0), ml = T(0), pp = T(0), pm = T(0);
    // normal stresses: 2 mu of the two cells (stored doubled: scaling by two
    // is exact, so this equals doubling mu pp + mu pm afterwards)
    if (!za || DIAG) {
        mh = ld(C.mu2_c + X.c_h);
        ml = ld(C.mu2_c + X.c_l);
    }
    if (!za) {
        pp = ga(X.a_p);
        pm = ga(X.a_m);
        N = mh * pp;
        N = fma(ml, pm, N);
    }
    if (DIAG) dsum = mh + ml;
    T lh = T(0), ll = T(0);
    if (BULK) {   // a compile-time switch: the plain form issues no bulk work
        lh = ld(C.lam_c + X.c_h);
        ll = ld(C.lam_c + X.c_l);
        if (!za) {
            N = fma(lh, pp, N);
            N = fma(ll, pm, N);
        }
        if (DIAG) dsum += lh + ll;
    }
#pragma unroll
    for (int j = 0; j < DIM - 1; ++j) {
        const int B = trans_axis(DIM, A, j);
        const int P = A + B - 1;   // edge pair index of {A, B}
        const bool zb = (ZM >> B) & 1;   // folds to a constant once j is unrolled
        if (za && zb && !DIAG) continue;
        const T mlo = ld(C.mu_e[P] + X.e_lo[j]);
        const T mhi = ld(C.mu_e[P] + X.e_hi[j]);
        if (!zb) {
            // d phi_B / dx_A on the two edges: B-faces in A-cells q[A] and q[A]-1
            const T xlo = gb(B, X.b_q[j]) - gb(B, X.b_r0[j]);
            const T xhi = gb(B, X.b_qe[j]) - gb(B, X.b_r2[j]);
            if (!za && sizeof(T) == 8) {
                // one add each; a wall neighbour contributes a selected zero
                // (no negated copy of xlo is formed: in FP64 that costs an
                // instruction of its own on the FP64 pipe, 18 -> 16 per face)
                const T shi = xhi + (X.whi[j] ? T(0) : ga(X.a_bp[j]));
                const T slo = (X.wlo[j] ? T(0) : ga(X.a_bm[j])) - xlo;
                N = fma(mhi, shi, N);
                N = fma(mlo, slo, N);
            } else if (!za) {   // FP32: conditional adds (measured a little faster there)
                T shi = xhi, slo = -xlo;
                if (!X.whi[j]) shi += ga(X.a_bp[j]);
                if (!X.wlo[j]) slo += ga(X.a_bm[j]);
                N = fma(mhi, shi, N);
                N = fma(mlo, slo, N);
            } else {
                N = fma(mhi, xhi, N);
                N = fma(-mlo, xlo, N);
            }
        } else if (!za) {
            const T shi = X.whi[j] ? T(0) : ga(X.a_bp[j]);
            const T slo = X.wlo[j] ? T(0) : ga(X.a_bm[j]);
            N = fma(mhi, shi, N);
            N = fma(mlo, slo, N);
        }
        if (DIAG) {   // explicit fmas: the same rounding in every kernel that inlines this
            dsum = fma(X.whi[j] ? T(2) : T(1), mhi, dsum);
            dsum = fma(X.wlo[j] ? T(2) : T(1), mlo, dsum);
        }
        if (BULK && !zb) {   // B-divergence of the cells q (hi) and q - e_A (lo)
            N = fma(lh, gb(B, X.b_qe[j]) - gb(B, X.b_q[j]), N);
            N = fma(-ll, gb(B, X.b_r2[j]) - gb(B, X.b_r0[j]), N);
        }
    }
    return N;
}

// Coordinate accessors: pa(r) reads phi_A at the A-face r (any storage, e.g.
// shared memory), pb(B, i) reads phi_B at the global index i.
template <int DIM, int A, typename T, bool DIAG, bool BULK, typename AI, typename GA, typename PB>
__device__ __forceinline__ T visc_offdiag_acc(const Geom& g, const Coef<T>& C, const int q[3],
                                              const AI& aidx, const GA& ga, const PB& pb, T& dsum) {
    Nbr X;
    nbr_coord<DIM, A>(g, q, aidx, X);
    return visc_offdiag_tab<DIM, A, T, DIAG, BULK>(C, X, ga, pb, dsum);
}

// phi a packed global vector: the strided index table
template <int DIM, int A, typename T, typename TV, bool DIAG, bool BULK = false, int ZM = 0>
__device__ __forceinline__ T visc_offdiag_h2(const Geom& g, const Coef<T>& C, const int q[3],
                                             const TV* phi, T& dsum) {
    Nbr X;
    nbr_lin<DIM, A>(g, q, X);
    return visc_offdiag_tab<DIM, A, T, DIAG, BULK, ZM>(
        C, X, [&](int i) { return T(phi[i]); }, [&](int, int i) { return T(phi[i]); }, dsum);
}

template <int DIM, typename T, typename TV, bool DIAG, bool BULK = false>
__device__ __forceinline__ T visc_offdiag_any(int a, const Geom& g, const Coef<T>& C,
                                              const int q[3], const TV* phi, T& dsum) {
    if (a == 0) return visc_offdiag_h2<DIM, 0, T, TV, DIAG, BULK>(g, C, q, phi, dsum);
    if (a == 1) return visc_offdiag_h2<DIM, 1, T, TV, DIAG, BULK>(g, C, q, phi, dsum);
    return visc_offdiag_h2<DIM, DIM == 3 ? 2 : 1, T, TV, DIAG, BULK>(g, C, q, phi, dsum);
}

// Off-diagonal part of h^2 L_rho at cell q: Nc = sum_a (beta_hi phi[+a] +
// beta_lo phi[-a]) and bsum = sum_a (beta_hi + beta_lo), so that
// h^2 (L_rho phi)_q = Nc - bsum phi_q (beta = 0 on wall faces).
template <int DIM, typename T, typename PC>
__device__ __forceinline__ T poisson_offdiag_acc(const Geom& g, const Coef<T>& C, const int q[3],
                                                 const PC& pc, T& bsum) {
    // pc(r): phi at cell r
    T N = T(0);
    bsum = T(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int fh[3] = {q[0], q[1], q[2]};
        fh[a] = g.per[a] ? wrapm(q[a] + 1, g.n[a]) : q[a] + 1;
        const T bh = ld(C.beta + fidx(g, a, fh));
        const T bl = ld(C.beta + fidx(g, a, q));
        int ch[3] = {q[0], q[1], q[2]};
        int cl[3] = {q[0], q[1], q[2]};
        ch[a] = g.per[a] ? wrapm(q[a] + 1, g.n[a]) : min(q[a] + 1, g.n[a] - 1);
        cl[a] = g.per[a] ? wrapm(q[a] - 1, g.n[a]) : max(q[a] - 1, 0);
        N = fma(bh, pc(ch), N);
        N = fma(bl, pc(cl), N);
        bsum += bh + bl;
    }
    return N;
}

// The same sum for phi a packed cell vector (c = cidx(q)), from one base
// index per array and constant strides; the periodic seam and the clamped
// wall neighbour (itself, with beta = 0) are branch-free corrections.  Same
// arithmetic order as poisson_offdiag_acc, so the same rounding.
template <int DIM, typename T, typename TV>
__device__ __forceinline__ T poisson_offdiag_h2(const Geom& g, const Coef<T>& C, const int q[3],
                                                int c, const TV* phi, T& bsum) {
    T N = T(0);
    bsum = T(0);
    int sc = 1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const int na = g.n[a];
        const bool top = q[a] == na - 1, bot = q[a] == 0;
        const int sf = a == 0 ? 1 : (a == 1 ? g.fe[a][0] : g.fe[a][0] * g.fe[a][1]);
        const int fl = fidx(g, a, q);
        const int fh = STK_IDX(fl + ((g.per[a] && top) ? 1 - na : 1) * sf, g.nvel, 1);
        const int ch = STK_IDX(c + (top ? (g.per[a] ? 1 - na : 0) : 1) * sc, g.ncell, 2);
        const int cl = STK_IDX(c - (bot ? (g.per[a] ? 1 - na : 0) : 1) * sc, g.ncell, 2);
        const T bh = ld(C.beta + fh);
        const T bl = ld(C.beta + fl);
        N = fma(bh, T(phi[ch]), N);
        N = fma(bl, T(phi[cl]), N);
        bsum += bh + bl;
        sc *= na;
    }
    return N;
}

// (L_rho phi) at cell q and its diagonal; beta = 0 on wall faces.
template <int DIM, typename T, typename TV>
__device__ __forceinline__ T poisson_cell(const Geom& g, const Coef<T>& C, const int q[3],
                                          const TV* phi, T& diag) {
    const T ih2 = gih2<T>(g);
    const T pc = T(phi[cidx(g, q)]);
    T L = T(0);
    diag = T(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int fh[3] = {q[0], q[1], q[2]};
        fh[a] = g.per[a] ? wrapm(q[a] + 1, g.n[a]) : q[a] + 1;
        const T bh = ld(C.beta + fidx(g, a, fh));
        const T bl = ld(C.beta + fidx(g, a, q));
        int ch[3] = {q[0], q[1], q[2]};
        int cl[3] = {q[0], q[1], q[2]};
        ch[a] = g.per[a] ? wrapm(q[a] + 1, g.n[a]) : min(q[a] + 1, g.n[a] - 1);
        cl[a] = g.per[a] ? wrapm(q[a] - 1, g.n[a]) : max(q[a] - 1, 0);
        L += ih2 * (bh * (T(phi[cidx(g, ch)]) - pc) - bl * (pc - T(phi[cidx(g, cl)])));
        diag -= ih2 * (bh + bl);
    }
    return L;
}

// ---------------------------------------------------------- per-point updates
// Gauss-Seidel update phi += D^{-1}(rhs - A phi) of the interior A-face q
// (App. C, omega = 1) with the stored inverse diagonal of the level's
// precision (FP32: the FP64 inverse rounded): a load in place of forming
// the diagonal and dividing.
template <typename T>
__device__ __forceinline__ T vel_gs_value(const Geom& g, const Coef<T>& C, int f, T N, const T* rhs) {
    const T num = fma(gih2<T>(g), N, rhs[f]);
    return num * ld(C.invd_u + f);
}

template <int DIM, int A, typename T, bool BULK = false, int ZM = 0>
__device__ __forceinline__ void vel_gs_point(const Geom& g, const Coef<T>& C, const int q[3],
                                             T* phi, const T* rhs) {
    T dsum;
    const T N = visc_offdiag_h2<DIM, A, T, T, false, BULK, ZM>(g, C, q, phi, dsum);
    const int f = fidx(g, A, q);
    phi[f] = vel_gs_value<T>(g, C, f, N, rhs);
}

template <int DIM, typename T, bool BULK = false>
__device__ __forceinline__ T vel_res_point(int a, const Geom& g, const Coef<T>& C, const int q[3],
                                           const T* phi, const T* rhs) {
    constexpr bool F32 = sizeof(T) == 4;
    const int f = fidx(g, a, q);
    T dsum;
    const T N = visc_offdiag_any<DIM, T, T, F32, BULK>(a, g, C, q, phi, dsum);
    const T ih2 = gih2<T>(g);
    const T diag = F32 ? fma(ih2, dsum, ld(C.alpha + f)) : ld(C.diag_u + f);
    return fma(-diag, phi[f], fma(ih2, N, rhs[f]));
}

// 6-point (2D) / 12-point (3D) restriction to the interior coarse A-face Q:
// 1/4 (1/8) on the coincident fine faces, 1/8 (1/16) on their neighbours.
template <int DIM, int A, typename T>
__device__ __forceinline__ T vel_restrict_point(const Geom& gf, const int Q[3],
                                                const T* res) {
    using TR = Trans<DIM, A>;
    const T wt = DIM == 3 ? T(0.25) : T(0.5);
    T acc = T(0);
#pragma unroll
    for (int s = -1; s <= 1; ++s) {
        const T w = (s == 0 ? T(0.5) : T(0.25)) * wt;
#pragma unroll
        for (int t0 = 0; t0 < 2; ++t0)
#pragma unroll
            for (int t1 = 0; t1 < (TR::n == 2 ? 2 : 1); ++t1) {
                int q[3] = {2 * Q[0], 2 * Q[1], DIM == 3 ? 2 * Q[2] : Q[2]};
                q[A] = step(gf, A, q[A], s);
                q[TR::b0] += t0;
                if (TR::n == 2) q[TR::b1] += t1;
                acc = fma(w, res[fidx(gf, A, q)], acc);
            }
    }
    return acc;
}

// transverse weights of the face prolongation along axis b for fine cell j:
// 3/4 on coarse cell J = j/2, 1/4 on the nearer neighbour; a neighbour across
// a wall is a ghost -phi (no-slip) or +phi (free-slip) folded onto J.  With
// `half` both weights are halved (the normal-direction average of an odd
// fine face folded in).  The weights are selected constants of type T (no
// conversions, no multiplies).
template <typename T>
__device__ __forceinline__ void prolong_transverse(const Geom& gc, int b, int j, bool half, int& J,
                                                   int& nb, T& wo, T& wn) {
    J = j >> 1;
    nb = (j & 1) ? J + 1 : J - 1;
    wo = half ? T(0.375) : T(0.75);
    wn = half ? T(0.125) : T(0.25);
    if (nb < 0 || nb >= gc.n[b]) {
        if (gc.per[b]) {
            nb = wrapm(nb, gc.n[b]);
        } else {
            const bool noslip = (nb < 0 ? gc.bclo[b] : gc.bchi[b]) == NOSLIP;
            wo = noslip ? (half ? T(0.25) : T(0.5)) : (half ? T(0.5) : T(1));
            wn = T(0);
            nb = J;
        }
    }
}

// (P phi_c) at the interior fine A-face q (App. C face prolongation): the
// coincident coarse faces (even q_A) or the mean of the two enclosing ones
// (odd q_A), interpolated transversally with the weights above.
template <int DIM, int A, typename T>
__device__ __forceinline__ T vel_prolong_point(const Geom& gc, const int q[3],
                                               const T* pc) {
    using TR = Trans<DIM, A>;
    const int ca0 = q[A] >> 1;
    const bool odd = q[A] & 1;
    int ca1 = ca0 + 1;
    if (gc.per[A] && ca1 >= gc.n[A]) ca1 -= gc.n[A];
    int J0, N0, J1 = 0, N1 = 0;
    T wo0, wn0, wo1 = T(1), wn1 = T(0);
    prolong_transverse<T>(gc, TR::b0, q[TR::b0], odd, J0, N0, wo0, wn0);
    if (TR::n == 2) prolong_transverse<T>(gc, TR::b1, q[TR::b1], false, J1, N1, wo1, wn1);
    // coarse value at transverse position (j0, j1): one face (even) or the
    // sum of the two along A (odd; the 1/2 is in wo0, wn0)
    auto at = [&](int j0, int j1) -> T {
        int Q[3] = {0, 0, DIM == 3 ? 0 : q[2]};
        Q[A] = ca0;
        Q[TR::b0] = j0;
        if (TR::n == 2) Q[TR::b1] = j1;
        T v = pc[fidx(gc, A, Q)];
        if (odd) {
            Q[A] = ca1;
            v += pc[fidx(gc, A, Q)];
        }
        return v;
    };
    if (TR::n == 2) {
        const T t0 = fma(wn1, at(J0, N1), wo1 * at(J0, J1));
        const T t1 = fma(wn1, at(N0, N1), wo1 * at(N0, J1));
        return fma(wn0, t1, wo0 * t0);
    }
    return fma(wn0, at(N0, 0), wo0 * at(J0, 0));
}

template <typename T>
__device__ __forceinline__ T cell_gs_update(const Geom& g, const Coef<T>& C, int c, T N,
                                            const T* rhs) {
    const T num = fma(-gih2<T>(g), N, rhs[c]);   // (rhs - off-diagonal part) / diag
    return num * ld(C.invd_p + c);
}

template <int DIM, typename T, typename PC>
__device__ __forceinline__ T cell_gs_value(const Geom& g, const Coef<T>& C, const int q[3],
                                           const PC& pc, const T* rhs) {
    T bsum;
    const T N = poisson_offdiag_acc<DIM, T>(g, C, q, pc, bsum);
    return cell_gs_update<T>(g, C, cidx(g, q), N, rhs);
}

template <int DIM, typename T, bool Z = false>
__device__ __forceinline__ void cell_gs_point(const Geom& g, const Coef<T>& C, const int q[3],
                                              T* phi, const T* rhs) {
    const int c = cidx(g, q);
    if (Z) {   // every neighbour zero: no beta needed either
        phi[c] = cell_gs_update<T>(g, C, c, T(0), rhs);
        return;
    }
    T bsum;
    const T N = poisson_offdiag_h2<DIM, T, T>(g, C, q, c, phi, bsum);
    phi[c] = cell_gs_update<T>(g, C, c, N, rhs);
}

template <int DIM, typename T>
__device__ __forceinline__ T cell_res_point(const Geom& g, const Coef<T>& C, const int q[3],
                                            const T* phi, const T* rhs) {
    const int c = cidx(g, q);
    T bsum;
    const T N = poisson_offdiag_h2<DIM, T, T>(g, C, q, c, phi, bsum);
    return fma(-gih2<T>(g), fma(-bsum, T(phi[c]), N), rhs[c]);
}

template <int DIM, typename T>
__device__ __forceinline__ T cell_restrict_point(const Geom& gf, const int Q[3],
                                                 const T* res) {
    T s = T(0);
#pragma unroll
    for (int dz = 0; dz < (DIM == 3 ? 2 : 1); ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                int q[3] = {2 * Q[0] + dx, 2 * Q[1] + dy, (DIM == 3 ? 2 * Q[2] : Q[2]) + dz};
                s += res[cidx(gf, q)];
            }
    return s * (DIM == 3 ? T(0.125) : T(0.25));
}

}  // namespace st
}  // namespace stk
