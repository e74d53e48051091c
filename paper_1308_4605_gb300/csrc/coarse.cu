// Coarse levels of the V-cycles (App. C) in one single-block launch.
//
// Below about 4096 cells a level's smoothing, residual and transfer kernels
// are a few blocks each and their run time is launch latency.  This kernel
// runs the whole lower part of a V-cycle -- every level from the given one
// down to the coarsest (2 cells along the shortest axis) and back up -- in
// one block of 1024 threads, with __syncthreads() between the stages.  The
// arithmetic is that of the grid-wide kernels: the same per-point functions
// of stencil.cuh in the same stage order (nu pre-sweeps, residual,
// restriction, recursion, prolongation, nu post-sweeps; ncoarse sweeps on the
// coarsest level; zero initial guess on every level).
#include "stencil.cuh"

namespace stk {
namespace {

using namespace st;
constexpr int CT = 1024;

template <int DIM, typename T, bool BULK>
__device__ void c_vel_sweeps(const Geom& g, const Coef<T>& C, int nsweep, T* phi, const T* rhs) {
    for (int it = 0; it < nsweep; ++it)
#pragma unroll
        for (int a = 0; a < DIM; ++a)
            for (int par = 0; par < 2; ++par) {
                const int nt = ((g.fe[a][0] + 1) >> 1) * g.fe[a][1] * g.fe[a][2];
                for (int t = threadIdx.x; t < nt; t += CT) {
                    int q[3];
                    if (!decode_face_colour(g, a, par, t, q) || wall_face(g, a, q)) continue;
                    if (a == 0) vel_gs_point<DIM, 0, T, BULK>(g, C, q, phi, rhs);
                    else if (a == 1) vel_gs_point<DIM, 1, T, BULK>(g, C, q, phi, rhs);
                    else vel_gs_point<DIM, DIM == 3 ? 2 : 1, T, BULK>(g, C, q, phi, rhs);
                }
                __syncthreads();
            }
}

template <int DIM, typename T>
__device__ void c_cell_sweeps(const Geom& g, const Coef<T>& C, int nsweep, T* phi, const T* rhs) {
    const int nt = (g.n[0] >> 1) * g.n[1] * g.n[2];
    for (int it = 0; it < nsweep; ++it)
        for (int par = 0; par < 2; ++par) {
            for (int t = threadIdx.x; t < nt; t += CT) {
                int q[3];
                decode_cell_colour(g, par, t, q);
                cell_gs_point<DIM, T>(g, C, q, phi, rhs);
            }
            __syncthreads();
        }
}

__device__ __forceinline__ void load_geom(Geom* dst, const Geom* src) {
    // cooperative copy of a level's geometry into shared memory
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(Geom) / sizeof(int)); i += CT) d[i] = s[i];
}

template <int DIM, typename T, bool BULK>
__global__ void __launch_bounds__(CT) k_coarse_vel(const CLevel<T>* __restrict__ Ls, int nlev,
                                                   const T* rhs0, T* phi0, int nu, int ncoarse) {
    pdl_entry();
    __shared__ Geom gsh[2];
    // down: pre-smoothing, residual, restriction
    for (int l = 0; l < nlev; ++l) {
        load_geom(&gsh[0], &Ls[l].g);
        if (l + 1 < nlev) load_geom(&gsh[1], &Ls[l + 1].g);
        __syncthreads();
        const Geom& g = gsh[0];
        const Coef<T> C = Ls[l].C;
        T* phi = l == 0 ? phi0 : Ls[l].phi_u;
        const T* rhs = l == 0 ? rhs0 : Ls[l].rhs_u;
        for (int t = threadIdx.x; t < g.nvel; t += CT) phi[t] = T(0);
        __syncthreads();
        if (l + 1 == nlev) {
            c_vel_sweeps<DIM, T, BULK>(g, C, ncoarse, phi, rhs);
            break;
        }
        c_vel_sweeps<DIM, T, BULK>(g, C, nu, phi, rhs);
        T* res = Ls[l].res_u;
        for (int t = threadIdx.x; t < g.nvel; t += CT) {
            int a = 0;
            while (a + 1 < DIM && t >= g.foff[a + 1]) ++a;
            int q[3];
            decode_face(g, a, t - g.foff[a], q);
            res[t] = wall_face(g, a, q) ? T(0) : vel_res_point<DIM, T, BULK>(a, g, C, q, phi, rhs);
        }
        __syncthreads();
        const Geom& gc = gsh[1];
        T* rc = Ls[l + 1].rhs_u;
        for (int t = threadIdx.x; t < gc.nvel; t += CT) {
            int a = 0;
            while (a + 1 < DIM && t >= gc.foff[a + 1]) ++a;
            int Q[3];
            decode_face(gc, a, t - gc.foff[a], Q);
            T v = T(0);
            if (!wall_face(gc, a, Q)) {
                if (a == 0) v = vel_restrict_point<DIM, 0, T>(g, Q, res);
                else if (a == 1) v = vel_restrict_point<DIM, 1, T>(g, Q, res);
                else v = vel_restrict_point<DIM, DIM == 3 ? 2 : 1, T>(g, Q, res);
            }
            rc[t] = v;
        }
        __syncthreads();
    }
    // up: prolongation and correction, post-smoothing
    for (int l = nlev - 2; l >= 0; --l) {
        load_geom(&gsh[0], &Ls[l].g);
        load_geom(&gsh[1], &Ls[l + 1].g);
        __syncthreads();
        const Geom& g = gsh[0];
        const Geom& gc = gsh[1];
        const Coef<T> C = Ls[l].C;
        T* phi = l == 0 ? phi0 : Ls[l].phi_u;
        const T* rhs = l == 0 ? rhs0 : Ls[l].rhs_u;
        const T* pc = Ls[l + 1].phi_u;
        for (int t = threadIdx.x; t < g.nvel; t += CT) {
            int a = 0;
            while (a + 1 < DIM && t >= g.foff[a + 1]) ++a;
            int q[3];
            decode_face(g, a, t - g.foff[a], q);
            if (wall_face(g, a, q)) continue;
            T v;
            if (a == 0) v = vel_prolong_point<DIM, 0, T>(gc, q, pc);
            else if (a == 1) v = vel_prolong_point<DIM, 1, T>(gc, q, pc);
            else v = vel_prolong_point<DIM, DIM == 3 ? 2 : 1, T>(gc, q, pc);
            phi[t] += v;
        }
        __syncthreads();
        c_vel_sweeps<DIM, T, BULK>(g, C, nu, phi, rhs);
    }
}

template <int DIM, typename T>
__global__ void __launch_bounds__(CT) k_coarse_cell(const CLevel<T>* __restrict__ Ls, int nlev,
                                                    const T* rhs0, T* phi0, int nu, int ncoarse) {
    pdl_entry();
    __shared__ Geom gsh[2];
    for (int l = 0; l < nlev; ++l) {
        load_geom(&gsh[0], &Ls[l].g);
        if (l + 1 < nlev) load_geom(&gsh[1], &Ls[l + 1].g);
        __syncthreads();
        const Geom& g = gsh[0];
        const Coef<T> C = Ls[l].C;
        T* phi = l == 0 ? phi0 : Ls[l].phi_p;
        const T* rhs = l == 0 ? rhs0 : Ls[l].rhs_p;
        for (int t = threadIdx.x; t < g.ncell; t += CT) phi[t] = T(0);
        __syncthreads();
        if (l + 1 == nlev) {
            c_cell_sweeps<DIM, T>(g, C, ncoarse, phi, rhs);
            break;
        }
        c_cell_sweeps<DIM, T>(g, C, nu, phi, rhs);
        T* res = Ls[l].res_p;
        for (int t = threadIdx.x; t < g.ncell; t += CT) {
            int q[3];
            decode_cell(g, t, q);
            res[t] = cell_res_point<DIM, T>(g, C, q, phi, rhs);
        }
        __syncthreads();
        const Geom& gc = gsh[1];
        T* rc = Ls[l + 1].rhs_p;
        for (int t = threadIdx.x; t < gc.ncell; t += CT) {
            int Q[3];
            decode_cell(gc, t, Q);
            rc[t] = cell_restrict_point<DIM, T>(g, Q, res);
        }
        __syncthreads();
    }
    for (int l = nlev - 2; l >= 0; --l) {
        load_geom(&gsh[0], &Ls[l].g);
        load_geom(&gsh[1], &Ls[l + 1].g);
        __syncthreads();
        const Geom& g = gsh[0];
        const Geom& gc = gsh[1];
        const Coef<T> C = Ls[l].C;
        T* phi = l == 0 ? phi0 : Ls[l].phi_p;
        const T* rhs = l == 0 ? rhs0 : Ls[l].rhs_p;
        const T* pc = Ls[l + 1].phi_p;
        for (int t = threadIdx.x; t < g.ncell; t += CT) {
            int q[3];
            decode_cell(g, t, q);
            int Q[3] = {q[0] >> 1, q[1] >> 1, DIM == 3 ? q[2] >> 1 : 0};
            phi[t] += pc[cidx(gc, Q)];
        }
        __syncthreads();
        c_cell_sweeps<DIM, T>(g, C, nu, phi, rhs);
    }
}

}  // namespace

template <typename T>
void launch_coarse_vcycle_vel(int dim, const CLevel<T>* L, int nlev, const T* rhs, T* phi, int nu,
                              int ncoarse, bool bulk, cudaStream_t s) {
    if (dim == 2) launch_pdl(bulk ? k_coarse_vel<2, T, true> : k_coarse_vel<2, T, false>, dim3(1), dim3(CT), s, L, nlev, rhs, phi, nu, ncoarse);
    else launch_pdl(bulk ? k_coarse_vel<3, T, true> : k_coarse_vel<3, T, false>, dim3(1), dim3(CT), s, L, nlev, rhs, phi, nu, ncoarse);
}

template <typename T>
void launch_coarse_vcycle_cell(int dim, const CLevel<T>* L, int nlev, const T* rhs, T* phi, int nu,
                               int ncoarse, cudaStream_t s) {
    if (dim == 2) launch_pdl(k_coarse_cell<2, T>, dim3(1), dim3(CT), s, L, nlev, rhs, phi, nu, ncoarse);
    else launch_pdl(k_coarse_cell<3, T>, dim3(1), dim3(CT), s, L, nlev, rhs, phi, nu, ncoarse);
}

template void launch_coarse_vcycle_vel<double>(int, const CLevel<double>*, int, const double*,
                                               double*, int, int, bool, cudaStream_t);
template void launch_coarse_vcycle_vel<float>(int, const CLevel<float>*, int, const float*, float*,
                                              int, int, bool, cudaStream_t);
template void launch_coarse_vcycle_cell<double>(int, const CLevel<double>*, int, const double*,
                                                double*, int, int, cudaStream_t);
template void launch_coarse_vcycle_cell<float>(int, const CLevel<float>*, int, const float*,
                                               float*, int, int, cudaStream_t);

}  // namespace stk
