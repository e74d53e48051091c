// The FP64 Stokes operator and the finest-level velocity residual evaluated
// through stresses (Sec. 3.1, Eq. div_stress): first the normal stresses at
// cells and the shear stresses on edges, each once, then the momentum rows
// as differences of stresses across each face.
//
// The per-face stencil (stencil.cuh) recomputes each edge stress for every
// face that touches the edge (four of them) and each normal stress for both
// faces of a cell.  On GB300 the FP64 operator is bound by the FP64 pipe, so
// computing each stress once (a few FP64 operations per cell and edge, then
// 6 to 7 per face) instead of about 20 per face is worth the extra stores
// and loads of the stress arrays.  Shear stresses are kept scaled by h
// (differences, not derivatives) and the momentum rows carry their 1/h^2;
// for the operator the cell values already include 1/h^2 and the pressure.
//
// Conventions as in stencil.cuh: wall faces hold the prescribed normal
// velocity (zero for the homogeneous problem); a no-slip wall's tangential
// derivative is one-sided, (u_first - 0)/(h/2), i.e. the difference 2 u_first;
// free-slip walls and edges on two walls carry zero shear stress (their edge
// viscosity is zero).
#include <type_traits>

#include "stencil.cuh"

namespace stk {
namespace {

using namespace st;
constexpr int ST = 256;

__device__ __forceinline__ void unflat(int t, const int e[3], int q[3]) {
    q[0] = t % e[0];
    const int r = t / e[0];
    q[1] = r % e[1];
    q[2] = r / e[1];
}

// Normal stresses tau_aa = 2 mu (u_a[c + e_a] - u_a[c]) (+ lam div u with bulk
// viscosity) and, when ycell is given, the continuity rows ycell_c = -(D u)_c
// (or bcell_c + (D u)_c).  PRES (the operator): the cell values are the full
// normal components of the stress divided by h, tau_aa / h^2 - p / h, so that
// a momentum row takes the pressure gradient and the 1/h^2 scaling of the
// normal stresses with them (two operations per cell instead of three per
// face).
template <int DIM, bool BULK, bool PRES>
__global__ void __launch_bounds__(ST) k_stress_cells(Geom g, Coef<double> C, const double* __restrict__ x,
                                                     const double* __restrict__ bcell,
                                                     double* __restrict__ ycell,
                                                     double* __restrict__ tau0, double* __restrict__ tau1,
                                                     double* __restrict__ tau2) {
    pdl_entry();
    const int t = blockIdx.x * ST + threadIdx.x;
    if (t >= g.ncell) return;
    int q[3];
    decode_cell(g, t, q);
    auto dif = [&](auto A) -> double {
        constexpr int a = decltype(A)::value;
        int qh[3] = {q[0], q[1], q[2]};
        qh[a] = step(g, a, q[a], 1);
        return x[fidx(g, a, qh)] - x[fidx(g, a, q)];
    };
    const double d0 = dif(std::integral_constant<int, 0>{});
    const double d1 = dif(std::integral_constant<int, 1>{});
    const double d2 = DIM == 3 ? dif(std::integral_constant<int, 2>{}) : 0.0;
    const double div = DIM == 3 ? d0 + d1 + d2 : d0 + d1;
    if (PRES) {
        const double m2 = ld(C.mu2_c + t) * g.ih2;
        double base = -g.ih * x[g.nvel + t];
        if (BULK) base = fma(ld(C.lam_c + t) * g.ih2, div, base);
        tau0[t] = fma(m2, d0, base);
        tau1[t] = fma(m2, d1, base);
        if (DIM == 3) tau2[t] = fma(m2, d2, base);
    } else {
        const double m2 = ld(C.mu2_c + t);
        const double lam = BULK ? ld(C.lam_c + t) : 0.0;
        tau0[t] = BULK ? fma(lam, div, m2 * d0) : m2 * d0;
        tau1[t] = BULK ? fma(lam, div, m2 * d1) : m2 * d1;
        if (DIM == 3) tau2[t] = BULK ? fma(lam, div, m2 * d2) : m2 * d2;
    }
    if (ycell) ycell[t] = bcell ? fma(g.ih, div, bcell[t]) : -g.ih * div;
}

// Difference of component C across an edge along axis E (the C-faces at
// E-cell indices q[E] and q[E] - 1), one-sided on a wall: (u_first - 0) /
// (h/2) and (0 - u_last) / (h/2) as differences 2 u_first and -2 u_last.
template <int C, int E>
__device__ __forceinline__ double edge_diff(const Geom& g, const int q[3], const double* x) {
    int hi[3] = {q[0], q[1], q[2]};
    int lo[3] = {q[0], q[1], q[2]};
    if (g.per[E]) {
        lo[E] = wrapm(q[E] - 1, g.n[E]);
        return x[fidx(g, C, hi)] - x[fidx(g, C, lo)];
    }
    if (q[E] == 0) return 2.0 * x[fidx(g, C, hi)];
    lo[E] = q[E] - 1;
    if (q[E] == g.n[E]) return -2.0 * x[fidx(g, C, lo)];
    return x[fidx(g, C, hi)] - x[fidx(g, C, lo)];
}

// Shear stress on the edges of pair P (axes A < B): mu_e (du_A/dx_B + du_B/dx_A)
// as differences.  On an A-wall the A-faces are wall faces (their stored
// values); free-slip walls and edges on two walls have mu_e = 0.
template <int P>
__global__ void __launch_bounds__(ST) k_stress_edges(Geom g, Coef<double> Cf, const double* __restrict__ x,
                                                     double* __restrict__ tau) {
    pdl_entry();
    constexpr int A = P == 2 ? 1 : 0;
    constexpr int B = P == 0 ? 1 : 2;
    const int t = blockIdx.x * ST + threadIdx.x;
    if (t >= g.esize[P]) return;
    int q[3];
    unflat(t, g.ee[P], q);
    const double m = ld(Cf.mu_e[P] + t);
    tau[t] = m * (edge_diff<A, B>(g, q, x) + edge_diff<B, A>(g, q, x));   // m = 0: zero
}

// Momentum row of the interior A-face q.  MODE 0 (cell values from PRES):
// y = alpha u - (div of the stress, pressure included) (or b - that);
// MODE 1: r = rhs - alpha u + L u / h^2.
template <int DIM, int A, int MODE>
__device__ __forceinline__ double face_row(const Geom& g, const Coef<double>& C, const int q[3], int f,
                                           const double* x, const double* tca, const double* te0,
                                           const double* te1, const double* te2, const double* bb) {
    int qm[3] = {q[0], q[1], q[2]};
    qm[A] = step(g, A, q[A], -1);
    const double tn = tca[cidx(g, q)] - tca[cidx(g, qm)];
    // MODE 0: L holds the shear part alone (differences across the face's
    // edges); MODE 1: normal and shear parts
    double L = tn;
    bool first = true;
#pragma unroll
    for (int Bx = 0; Bx < DIM; ++Bx) {
        if (Bx == A) continue;
        const int p = A + Bx - 1;
        const double* te = p == 0 ? te0 : (p == 1 ? te1 : te2);
        int qe[3] = {q[0], q[1], q[2]};
        qe[Bx] = g.per[Bx] ? wrapm(q[Bx] + 1, g.n[Bx]) : q[Bx] + 1;
        const double de = te[eidx(g, p, qe)] - te[eidx(g, p, q)];
        L = (MODE == 0 && first) ? de : L + de;
        first = false;
    }
    const double u = x[f];
    if (MODE == 0) {
        const double Lf = fma(g.ih2, L, tn);   // the stress divergence, -grad p included
        const double Mx = fma(ld(C.alpha + f), u, -Lf);
        return bb ? bb[f] - Mx : Mx;
    }
    return fma(g.ih2, L, fma(-ld(C.alpha + f), u, bb[f]));
}

template <int DIM, int MODE>
__global__ void __launch_bounds__(ST) k_stress_faces(Geom g, Coef<double> C, int s1, int s2,
                                                     const double* __restrict__ x,
                                                     const double* __restrict__ tc0,
                                                     const double* __restrict__ tc1,
                                                     const double* __restrict__ tc2,
                                                     const double* __restrict__ te0,
                                                     const double* __restrict__ te1,
                                                     const double* __restrict__ te2,
                                                     const double* __restrict__ bb,
                                                     double* __restrict__ y, int zl) {
    pdl_entry();
    const int a = blockIdx.x < s1 ? 0 : (blockIdx.x < s2 ? 1 : 2);
    const int t = (blockIdx.x - (a == 0 ? 0 : a == 1 ? s1 : s2)) * ST + threadIdx.x;
    if (a >= DIM || t >= g.fsize[a]) return;
    int q[3];
    decode_face(g, a, t, q);
    const int f = g.foff[a] + t;
    if (wall_face(g, a, q) || (MODE == 1 && a == zl && (csum<DIM>(q) & 1))) {
        y[f] = 0.0;
        return;
    }
    double v;
    if (a == 0) v = face_row<DIM, 0, MODE>(g, C, q, f, x, tc0, te0, te1, te2, bb);
    else if (a == 1) v = face_row<DIM, 1, MODE>(g, C, q, f, x, tc1, te0, te1, te2, bb);
    else v = face_row<DIM, DIM == 3 ? 2 : 1, MODE>(g, C, q, f, x, tc2, te0, te1, te2, bb);
    y[f] = v;
}

inline int nb(long long n) { return (int)((n + ST - 1) / ST); }

template <bool PRES>
void stress_pass(const Geom& g, Coef<double> C, const StressWork& W, const double* x,
                 const double* bcell, double* ycell, cudaStream_t s) {
    const bool bulk = C.lam_c != nullptr;
    if (g.dim == 2)
        launch_pdl(bulk ? k_stress_cells<2, true, PRES> : k_stress_cells<2, false, PRES>, dim3(nb(g.ncell)),
                   dim3(ST), s, g, C, x, bcell, ycell, W.tc[0], W.tc[1], W.tc[2]);
    else
        launch_pdl(bulk ? k_stress_cells<3, true, PRES> : k_stress_cells<3, false, PRES>, dim3(nb(g.ncell)),
                   dim3(ST), s, g, C, x, bcell, ycell, W.tc[0], W.tc[1], W.tc[2]);
    launch_pdl(k_stress_edges<0>, dim3(nb(g.esize[0])), dim3(ST), s, g, C, x, W.te[0]);
    if (g.dim == 3) {
        launch_pdl(k_stress_edges<1>, dim3(nb(g.esize[1])), dim3(ST), s, g, C, x, W.te[1]);
        launch_pdl(k_stress_edges<2>, dim3(nb(g.esize[2])), dim3(ST), s, g, C, x, W.te[2]);
    }
}

template <int MODE>
void face_pass(const Geom& g, Coef<double> C, const StressWork& W, const double* x, const double* bb,
               double* y, int zl, cudaStream_t s) {
    const int s1 = nb(g.fsize[0]), s2 = s1 + nb(g.fsize[1]);
    const int total = s2 + (g.dim == 3 ? nb(g.fsize[2]) : 0);
    const double *tc0 = W.tc[0], *tc1 = W.tc[1], *tc2 = W.tc[2];
    const double *te0 = W.te[0], *te1 = W.te[1], *te2 = W.te[2];
    if (g.dim == 2)
        launch_pdl(k_stress_faces<2, MODE>, dim3(total), dim3(ST), s, g, C, s1, total, x, tc0, tc1, tc2,
                   te0, te1, te2, bb, y, zl);
    else
        launch_pdl(k_stress_faces<3, MODE>, dim3(total), dim3(ST), s, g, C, s1, s2, x, tc0, tc1, tc2,
                   te0, te1, te2, bb, y, zl);
}

}  // namespace

void launch_stokes_matvec_stress(const Geom& g, Coef<double> C, const StressWork& W, const double* x,
                                 const double* b, double* y, cudaStream_t s) {
    stress_pass<true>(g, C, W, x, b ? b + g.nvel : nullptr, y + g.nvel, s);
    face_pass<0>(g, C, W, x, b, y, -1, s);
}

void launch_vel_residual_stress(const Geom& g, Coef<double> C, const StressWork& W, const double* phi,
                                const double* rhs, double* res, bool after_sweep, cudaStream_t s) {
    stress_pass<false>(g, C, W, phi, nullptr, nullptr, s);
    face_pass<1>(g, C, W, phi, rhs, res, after_sweep ? g.dim - 1 : -1, s);
}

STK_OOB_READER(stress)

}  // namespace stk
