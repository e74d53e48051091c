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
//
// When the work vectors of these levels (phi, rhs and residual of each) fit
// in shared memory, the SMEM variant keeps them there: the kernel is a chain
// of about a hundred dependent stages, and each stage then waits on shared-
// memory instead of L2 latency.  Only the level's right-hand side is read
// from, and its solution written to, global memory; coefficients stay in
// global memory (read-only, cached).
#include "stencil.cuh"
#include "../../include/stokes.h"

#include <algorithm>

namespace stk {
namespace {

using namespace st;
constexpr int CT = 1024;
constexpr int CMAXL = 16;

// shared-memory layout of the SMEM variant: level l's phi at off[l], its rhs
// at off[l] + n_l and its residual at off[l] + 2 n_l (n_l = faces or cells)
struct SmemLevels {
    int off[CMAXL];
    int n[CMAXL];
};

// Barrier policies.  BlockSync: one block of CT threads, __syncthreads()
// between stages (the single-block kernel).  GridSync: every block of a
// cooperative launch, a grid-wide barrier between stages (the persistent
// multi-block kernel); each wait is bounded by a clock64() budget, after
// which the barrier writes STK_ERR_TIMEOUT to *status and every block
// returns at its next barrier, so a stalled launch ends instead of hanging.
// first() / end(): the points [first, end) of an array of `total` points
// that this thread visits (stride nth()).  A stacked batch (nsl instances
// along the slowest axis of every array) is run by one block per instance,
// each on its own contiguous share; otherwise the block takes every point.
struct BlockSync {
    __device__ __forceinline__ int tid() const { return threadIdx.x; }
    __device__ __forceinline__ int nth() const { return CT; }
    __device__ __forceinline__ int first(int total, int nsl) const {
        return nsl > 1 ? int(blockIdx.x) * (total / nsl) + int(threadIdx.x) : int(threadIdx.x);
    }
    __device__ __forceinline__ int end(int total, int nsl) const {
        return nsl > 1 ? (int(blockIdx.x) + 1) * (total / nsl) : total;
    }
    __device__ __forceinline__ bool sync() const {
        __syncthreads();
        return true;
    }
};

struct GridSync {
    unsigned* bar;        // [0] arrivals, [1] generation (zeroed before the launch)
    long long budget;     // clock64() cycles one wait may last (read from device memory at launch)
    int* status;          // 0, or STK_ERR_TIMEOUT once a wait ran out
    __device__ __forceinline__ int tid() const { return blockIdx.x * CT + threadIdx.x; }
    __device__ __forceinline__ int nth() const { return gridDim.x * CT; }
    // never used on a stacked batch: every block shares every point
    __device__ __forceinline__ int first(int, int) const { return tid(); }
    __device__ __forceinline__ int end(int total, int) const { return total; }
    // Sense-counting grid barrier: the block's writes are ordered before its
    // arrival (bar.sync, then a device-scope fence by thread 0), the last
    // block to arrive resets the count and advances the generation, the
    // others wait for the generation to change; the fence after the wait
    // orders the reads that follow.  false: a wait ran out (here or in
    // another block); the caller returns.
    __device__ bool sync() const {
        __shared__ int ok;
        __syncthreads();
        if (threadIdx.x == 0) {
            volatile unsigned* gen = bar + 1;
            volatile int* st = status;
            const unsigned g0 = *gen;
            __threadfence();
            int res = 1;
            if (atomicAdd(bar, 1u) + 1u == gridDim.x) {
                bar[0] = 0u;
                __threadfence();
                atomicAdd(bar + 1, 1u);
            } else {
                const long long t0 = clock64();
                while (*gen == g0) {
                    if (*st != 0 || clock64() - t0 > budget) {
                        atomicCAS(status, 0, STK_ERR_TIMEOUT);
                        res = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
            if (*st != 0) res = 0;
            ok = res;
        }
        __syncthreads();
        return ok != 0;
    }
};

// ClusterSync: the CTAs of one thread-block cluster (the whole grid is one
// cluster of at most 16 CTAs, resident together on one GPC) with the
// hardware cluster barrier between stages.  The stages exchange data through
// global memory written on other SMs of the cluster: the arrive has release
// and the wait acquire semantics at cluster scope, which order every
// thread's writes before the barrier with the reads after it.  Every CTA
// passes the same barriers and waits on nothing outside its own launch.
struct ClusterSync {
    __device__ __forceinline__ int tid() const { return blockIdx.x * CT + threadIdx.x; }
    __device__ __forceinline__ int nth() const { return gridDim.x * CT; }
    __device__ __forceinline__ int first(int, int) const { return tid(); }
    __device__ __forceinline__ int end(int total, int) const { return total; }
    __device__ __forceinline__ bool sync() const {
        asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                     "barrier.cluster.wait.acquire.aligned;" ::: "memory");
        return true;
    }
};

template <int DIM, typename T, bool BULK, typename SY>
__device__ bool c_vel_sweeps(const SY& S, const Geom& g, const Coef<T>& C, int nsweep, T* phi,
                             const T* rhs) {
    for (int it = 0; it < nsweep; ++it)
#pragma unroll
        for (int a = 0; a < DIM; ++a)
            for (int par = 0; par < 2; ++par) {
                const int nt = ((g.fe[a][0] + 1) >> 1) * g.fe[a][1] * g.fe[a][2];
                const int te = S.end(nt, g.nsl);
                for (int t = S.first(nt, g.nsl); t < te; t += S.nth()) {
                    int q[3];
                    if (!decode_face_colour(g, a, par, t, q) || wall_face(g, a, q)) continue;
                    if (a == 0) vel_gs_point<DIM, 0, T, BULK>(g, C, q, phi, rhs);
                    else if (a == 1) vel_gs_point<DIM, 1, T, BULK>(g, C, q, phi, rhs);
                    else vel_gs_point<DIM, DIM == 3 ? 2 : 1, T, BULK>(g, C, q, phi, rhs);
                }
                if (!S.sync()) return false;
            }
    return true;
}

template <int DIM, typename T, typename SY>
__device__ bool c_cell_sweeps(const SY& S, const Geom& g, const Coef<T>& C, int nsweep, T* phi,
                              const T* rhs) {
    const int nt = (g.n[0] >> 1) * g.n[1] * g.n[2];
    const int te = S.end(nt, g.nsl);
    for (int it = 0; it < nsweep; ++it)
        for (int par = 0; par < 2; ++par) {
            for (int t = S.first(nt, g.nsl); t < te; t += S.nth()) {
                int q[3];
                decode_cell_colour(g, par, t, q);
                cell_gs_point<DIM, T>(g, C, q, phi, rhs);
            }
            if (!S.sync()) return false;
        }
    return true;
}

// phi = S rhs with S stored column-major (st[i * n + j] = S_ji): each thread
// forms whole rows, summing over i in increasing order
template <typename T, typename SY>
__device__ void smat_apply(const SY& S, const T* __restrict__ st, int n, const T* rhs, T* phi) {
    for (int j = S.tid(); j < n; j += S.nth()) {
        T acc = T(0);
        for (int i = 0; i < n; ++i) acc = fma(st[(size_t)i * n + j], rhs[i], acc);
        phi[j] = acc;
    }
}

__device__ __forceinline__ void load_geom(Geom* dst, const Geom* src) {
    // cooperative copy of a level's geometry into shared memory
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(Geom) / sizeof(int)); i += CT) d[i] = s[i];
}

// Work vectors of level l: shared memory (SMEM) or the level's own arrays,
// level 0's right-hand side and solution being the caller's.
template <typename T, bool SMEM, bool VEL>
struct Vecs {
    const CLevel<T>* Ls;
    T* sm;
    const SmemLevels* sl;
    const T* rhs0;
    T* phi0;
    __device__ T* phi(int l) const {
        return SMEM ? sm + sl->off[l] : (l == 0 ? phi0 : (VEL ? Ls[l].phi_u : Ls[l].phi_p));
    }
    __device__ T* rhs(int l) const {
        return SMEM ? sm + sl->off[l] + sl->n[l]
                    : (l == 0 ? const_cast<T*>(rhs0) : (VEL ? Ls[l].rhs_u : Ls[l].rhs_p));
    }
    __device__ T* res(int l) const {
        return SMEM ? sm + sl->off[l] + 2 * sl->n[l] : (VEL ? Ls[l].res_u : Ls[l].res_p);
    }
};

// One velocity V-cycle (zero guess) over levels 0..nlev-1 of Ls.  Levels
// below lblock run with the barrier policy S; from level lblock on (lblock
// < nlev), block 0 alone runs the rest as a single-block V-cycle while the
// other blocks wait at the next barrier.  false: a barrier ran out.
template <int DIM, typename T, bool BULK, bool SMEM, typename SY>
__device__ bool vcycle_vel_body(const SY& S, Geom* gsh, const CLevel<T>* __restrict__ Ls, int nlev,
                                int lblock, const Vecs<T, SMEM, true> V, int nu, int ncoarse) {
    const int ltop = lblock < nlev ? lblock : nlev;
    // down: pre-smoothing, residual, restriction
    for (int l = 0; l < ltop; ++l) {
        load_geom(&gsh[0], &Ls[l].g);
        if (l + 1 < nlev) load_geom(&gsh[1], &Ls[l + 1].g);
        __syncthreads();
        const Geom& g = gsh[0];
        const Coef<T> C = Ls[l].C;
        T* phi = V.phi(l);
        const T* rhs = V.rhs(l);
        for (int a = 0; a < DIM; ++a)
            for (int t = S.first(g.fsize[a], g.nsl); t < S.end(g.fsize[a], g.nsl); t += S.nth())
                phi[g.foff[a] + t] = T(0);
        if (!S.sync()) return false;
        if (l + 1 == nlev) {   // coarsest level: the coarse solve, then up
            if (Ls[l].smat_u && Ls[l].smat_nc == ncoarse) smat_apply<T>(S, Ls[l].smat_u, g.nvel, rhs, phi);
            else if (!c_vel_sweeps<DIM, T, BULK>(S, g, C, ncoarse, phi, rhs)) return false;
            if (!S.sync()) return false;
            break;
        }
        if (!c_vel_sweeps<DIM, T, BULK>(S, g, C, nu, phi, rhs)) return false;
        T* res = V.res(l);
        for (int a = 0; a < DIM; ++a)
            for (int t = S.first(g.fsize[a], g.nsl); t < S.end(g.fsize[a], g.nsl); t += S.nth()) {
                int q[3];
                decode_face(g, a, t, q);
                // the black faces of the last component were just solved: zero residual
                const bool solved = nu > 0 && a == DIM - 1 && (csum<DIM>(q) & 1);
                res[g.foff[a] + t] = (wall_face(g, a, q) || solved)
                                         ? T(0)
                                         : vel_res_point<DIM, T, BULK>(a, g, C, q, phi, rhs);
            }
        if (!S.sync()) return false;
        const Geom& gc = gsh[1];
        T* rc = V.rhs(l + 1);
        for (int a = 0; a < DIM; ++a)
            for (int t = S.first(gc.fsize[a], gc.nsl); t < S.end(gc.fsize[a], gc.nsl); t += S.nth()) {
                int Q[3];
                decode_face(gc, a, t, Q);
                T v = T(0);
                if (!wall_face(gc, a, Q)) {
                    if (a == 0) v = vel_restrict_point<DIM, 0, T>(g, Q, res);
                    else if (a == 1) v = vel_restrict_point<DIM, 1, T>(g, Q, res);
                    else v = vel_restrict_point<DIM, DIM == 3 ? 2 : 1, T>(g, Q, res);
                }
                rc[gc.foff[a] + t] = v;
            }
        if (!S.sync()) return false;
    }
    if (ltop < nlev) {   // the coarse levels, one block
        if (blockIdx.x == 0) {
            const Vecs<T, false, true> Vb{Ls + ltop, nullptr, nullptr, V.rhs(ltop), V.phi(ltop)};
            vcycle_vel_body<DIM, T, BULK, false>(BlockSync{}, gsh, Ls + ltop, nlev - ltop, nlev - ltop, Vb,
                                                 nu, ncoarse);
        }
        if (!S.sync()) return false;
    }
    // up: prolongation and correction, post-smoothing
    for (int l = ltop - 1; l >= 0; --l) {
        if (l + 1 >= nlev) continue;
        load_geom(&gsh[0], &Ls[l].g);
        load_geom(&gsh[1], &Ls[l + 1].g);
        __syncthreads();
        const Geom& g = gsh[0];
        const Geom& gc = gsh[1];
        const Coef<T> C = Ls[l].C;
        T* phi = V.phi(l);
        const T* rhs = V.rhs(l);
        const T* pc = V.phi(l + 1);
        for (int a = 0; a < DIM; ++a)
            for (int t = S.first(g.fsize[a], g.nsl); t < S.end(g.fsize[a], g.nsl); t += S.nth()) {
                int q[3];
                decode_face(g, a, t, q);
                if (wall_face(g, a, q)) continue;
                T v;
                if (a == 0) v = vel_prolong_point<DIM, 0, T>(gc, q, pc);
                else if (a == 1) v = vel_prolong_point<DIM, 1, T>(gc, q, pc);
                else v = vel_prolong_point<DIM, DIM == 3 ? 2 : 1, T>(gc, q, pc);
                phi[g.foff[a] + t] += v;
            }
        if (!S.sync()) return false;
        if (!c_vel_sweeps<DIM, T, BULK>(S, g, C, nu, phi, rhs)) return false;
    }
    return true;
}

template <int DIM, typename T, bool SMEM, typename SY>
__device__ bool vcycle_cell_body(const SY& S, Geom* gsh, const CLevel<T>* __restrict__ Ls, int nlev,
                                 int lblock, const Vecs<T, SMEM, false> V, int nu, int ncoarse) {
    const int ltop = lblock < nlev ? lblock : nlev;
    for (int l = 0; l < ltop; ++l) {
        load_geom(&gsh[0], &Ls[l].g);
        if (l + 1 < nlev) load_geom(&gsh[1], &Ls[l + 1].g);
        __syncthreads();
        const Geom& g = gsh[0];
        const Coef<T> C = Ls[l].C;
        T* phi = V.phi(l);
        const T* rhs = V.rhs(l);
        for (int t = S.first(g.ncell, g.nsl); t < S.end(g.ncell, g.nsl); t += S.nth()) phi[t] = T(0);
        if (!S.sync()) return false;
        if (l + 1 == nlev) {
            if (Ls[l].smat_p && Ls[l].smat_nc == ncoarse) smat_apply<T>(S, Ls[l].smat_p, g.ncell, rhs, phi);
            else if (!c_cell_sweeps<DIM, T>(S, g, C, ncoarse, phi, rhs)) return false;
            if (!S.sync()) return false;
            break;
        }
        if (!c_cell_sweeps<DIM, T>(S, g, C, nu, phi, rhs)) return false;
        T* res = V.res(l);
        for (int t = S.first(g.ncell, g.nsl); t < S.end(g.ncell, g.nsl); t += S.nth()) {
            int q[3];
            decode_cell(g, t, q);
            res[t] = (nu > 0 && (csum<DIM>(q) & 1)) ? T(0) : cell_res_point<DIM, T>(g, C, q, phi, rhs);
        }
        if (!S.sync()) return false;
        const Geom& gc = gsh[1];
        T* rc = V.rhs(l + 1);
        for (int t = S.first(gc.ncell, gc.nsl); t < S.end(gc.ncell, gc.nsl); t += S.nth()) {
            int Q[3];
            decode_cell(gc, t, Q);
            rc[t] = cell_restrict_point<DIM, T>(g, Q, res);
        }
        if (!S.sync()) return false;
    }
    if (ltop < nlev) {
        if (blockIdx.x == 0) {
            const Vecs<T, false, false> Vb{Ls + ltop, nullptr, nullptr, V.rhs(ltop), V.phi(ltop)};
            vcycle_cell_body<DIM, T, false>(BlockSync{}, gsh, Ls + ltop, nlev - ltop, nlev - ltop, Vb, nu,
                                            ncoarse);
        }
        if (!S.sync()) return false;
    }
    for (int l = ltop - 1; l >= 0; --l) {
        if (l + 1 >= nlev) continue;
        load_geom(&gsh[0], &Ls[l].g);
        load_geom(&gsh[1], &Ls[l + 1].g);
        __syncthreads();
        const Geom& g = gsh[0];
        const Geom& gc = gsh[1];
        const Coef<T> C = Ls[l].C;
        T* phi = V.phi(l);
        const T* rhs = V.rhs(l);
        const T* pc = V.phi(l + 1);
        for (int t = S.first(g.ncell, g.nsl); t < S.end(g.ncell, g.nsl); t += S.nth()) {
            int q[3];
            decode_cell(g, t, q);
            int Q[3] = {q[0] >> 1, q[1] >> 1, DIM == 3 ? q[2] >> 1 : q[2]};
            phi[t] += pc[cidx(gc, Q)];
        }
        if (!S.sync()) return false;
        if (!c_cell_sweeps<DIM, T>(S, g, C, nu, phi, rhs)) return false;
    }
    return true;
}

// single block: every level from Ls[0] down, work vectors in shared memory
// when they fit (SMEM), else in global memory
template <int DIM, typename T, bool BULK, bool SMEM>
__global__ void __launch_bounds__(CT) k_coarse_vel(const CLevel<T>* __restrict__ Ls, int nlev,
                                                   const T* rhs0, T* phi0, int nu, int ncoarse) {
    pdl_entry();
    __shared__ Geom gsh[2];
    __shared__ SmemLevels sl;
    extern __shared__ __align__(16) unsigned char c_smem[];
    T* sm = reinterpret_cast<T*>(c_smem);
    if (SMEM) {
        if (threadIdx.x == 0) {
            int cur = 0;
            for (int l = 0; l < nlev; ++l) {
                sl.off[l] = cur;
                sl.n[l] = Ls[l].g.nvel;
                cur += 3 * sl.n[l];
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < sl.n[0]; t += CT) sm[sl.n[0] + t] = rhs0[t];
    }
    const Vecs<T, SMEM, true> V{Ls, sm, &sl, rhs0, phi0};
    vcycle_vel_body<DIM, T, BULK, SMEM>(BlockSync{}, gsh, Ls, nlev, nlev, V, nu, ncoarse);
    if (SMEM) {   // the solution of the first level back to global memory
        __syncthreads();
        for (int t = threadIdx.x; t < sl.n[0]; t += CT) phi0[t] = sm[t];
    }
}

template <int DIM, typename T, bool SMEM>
__global__ void __launch_bounds__(CT) k_coarse_cell(const CLevel<T>* __restrict__ Ls, int nlev,
                                                    const T* rhs0, T* phi0, int nu, int ncoarse) {
    pdl_entry();
    __shared__ Geom gsh[2];
    __shared__ SmemLevels sl;
    extern __shared__ __align__(16) unsigned char c_smem[];
    T* sm = reinterpret_cast<T*>(c_smem);
    if (SMEM) {
        if (threadIdx.x == 0) {
            int cur = 0;
            for (int l = 0; l < nlev; ++l) {
                sl.off[l] = cur;
                sl.n[l] = Ls[l].g.ncell;
                cur += 3 * sl.n[l];
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < sl.n[0]; t += CT) sm[sl.n[0] + t] = rhs0[t];
    }
    const Vecs<T, SMEM, false> V{Ls, sm, &sl, rhs0, phi0};
    vcycle_cell_body<DIM, T, SMEM>(BlockSync{}, gsh, Ls, nlev, nlev, V, nu, ncoarse);
    if (SMEM) {
        __syncthreads();
        for (int t = threadIdx.x; t < sl.n[0]; t += CT) phi0[t] = sm[t];
    }
}

// Stacked batches: block s runs instance s.  Lall holds, per instance, the
// descriptors of the levels handled here (stride lstride between instances):
// the geometry of one instance and its coefficients (face arrays copied
// instance by instance, cell and edge arrays in place), so the shared-memory
// variant runs unchanged on the instance's own vectors.  Only the right-hand
// side and the solution of the first level are moved between the stacked
// layout (each face component holds the instances one after another) and
// shared memory.
template <typename T>
__device__ __forceinline__ int stk_index(const Geom& gl, bool vel, int s, int nsl, int i) {
    if (!vel) return s * gl.ncell + i;
    int a = 0;
    while (a + 1 < gl.dim && i >= gl.foff[a + 1]) ++a;
    return nsl * gl.foff[a] + s * gl.fsize[a] + (i - gl.foff[a]);
}

template <int DIM, typename T, bool BULK, bool VEL>
__global__ void __launch_bounds__(CT) k_coarse_stk(const CLevel<T>* __restrict__ Lall, int lstride, int nlev,
                                                   const T* rhs0, T* phi0, int nu, int ncoarse) {
    pdl_entry();
    __shared__ Geom gsh[2];
    __shared__ SmemLevels sl;
    extern __shared__ __align__(16) unsigned char c_smem[];
    T* sm = reinterpret_cast<T*>(c_smem);
    const int s = blockIdx.x, nsl = gridDim.x;
    const CLevel<T>* Ls = Lall + (size_t)s * lstride;
    if (threadIdx.x == 0) {
        int cur = 0;
        for (int l = 0; l < nlev; ++l) {
            sl.off[l] = cur;
            sl.n[l] = VEL ? Ls[l].g.nvel : Ls[l].g.ncell;
            cur += 3 * sl.n[l];
        }
    }
    load_geom(&gsh[0], &Ls[0].g);
    __syncthreads();
    const int n0 = sl.n[0];
    for (int t = threadIdx.x; t < n0; t += CT) sm[n0 + t] = rhs0[stk_index<T>(gsh[0], VEL, s, nsl, t)];
    __syncthreads();
    if (VEL) {
        const Vecs<T, true, true> V{Ls, sm, &sl, rhs0, phi0};
        vcycle_vel_body<DIM, T, BULK, true>(BlockSync{}, gsh, Ls, nlev, nlev, V, nu, ncoarse);
    } else {
        const Vecs<T, true, false> V{Ls, sm, &sl, rhs0, phi0};
        vcycle_cell_body<DIM, T, true>(BlockSync{}, gsh, Ls, nlev, nlev, V, nu, ncoarse);
    }
    __syncthreads();
    load_geom(&gsh[0], &Ls[0].g);
    __syncthreads();
    for (int t = threadIdx.x; t < n0; t += CT) phi0[stk_index<T>(gsh[0], VEL, s, nsl, t)] = sm[t];
}

// instance-by-instance copy of a stacked face array (coarse-level
// coefficients of a stacked batch): dst[s * nvel + i] = src[stk_index(i)]
template <typename T>
__global__ void k_faces_by_instance(Geom gl, int nsl, const T* __restrict__ src, T* __restrict__ dst) {
    pdl_entry();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (t < gl.nvel) dst[(size_t)s * gl.nvel + t] = src[stk_index<T>(gl, true, s, nsl, t)];
}

// Persistent multi-block V-cycle (cooperative launch, every block resident):
// levels 0..lblock-1 of Ls as grid-wide stages separated by bounded grid
// barriers, the levels from lblock on by block 0 alone.  It replaces one
// kernel launch per colour and transfer on the middle levels, where a launch
// costs more than the stage's work.
template <int DIM, typename T, bool BULK>
__global__ void __launch_bounds__(CT) k_grid_vel(const CLevel<T>* __restrict__ Ls, int nlev, int lblock,
                                                 const T* rhs0, T* phi0, int nu, int ncoarse,
                                                 unsigned* bar, const long long* budget, int* status) {
    __shared__ Geom gsh[2];
    const GridSync S{bar, *budget, status};
    const Vecs<T, false, true> V{Ls, nullptr, nullptr, rhs0, phi0};
    vcycle_vel_body<DIM, T, BULK, false>(S, gsh, Ls, nlev, lblock, V, nu, ncoarse);
}

template <int DIM, typename T>
__global__ void __launch_bounds__(CT) k_grid_cell(const CLevel<T>* __restrict__ Ls, int nlev, int lblock,
                                                  const T* rhs0, T* phi0, int nu, int ncoarse,
                                                  unsigned* bar, const long long* budget, int* status) {
    __shared__ Geom gsh[2];
    const GridSync S{bar, *budget, status};
    const Vecs<T, false, false> V{Ls, nullptr, nullptr, rhs0, phi0};
    vcycle_cell_body<DIM, T, false>(S, gsh, Ls, nlev, lblock, V, nu, ncoarse);
}

// The same V-cycle as one thread-block cluster: levels 0..lblock-1 of Ls as
// stages separated by cluster barriers (a hardware barrier, much cheaper
// than a grid-wide one or a kernel boundary), the levels from lblock on by
// block 0 alone.  Meant for the middle levels, whose launches cost more than
// their work.
template <int DIM, typename T, bool BULK>
__global__ void __launch_bounds__(CT) k_cluster_vel(const CLevel<T>* __restrict__ Ls, int nlev, int lblock,
                                                    const T* rhs0, T* phi0, int nu, int ncoarse) {
    pdl_entry();
    __shared__ Geom gsh[2];
    const Vecs<T, false, true> V{Ls, nullptr, nullptr, rhs0, phi0};
    vcycle_vel_body<DIM, T, BULK, false>(ClusterSync{}, gsh, Ls, nlev, lblock, V, nu, ncoarse);
}

template <int DIM, typename T>
__global__ void __launch_bounds__(CT) k_cluster_cell(const CLevel<T>* __restrict__ Ls, int nlev, int lblock,
                                                     const T* rhs0, T* phi0, int nu, int ncoarse) {
    pdl_entry();
    __shared__ Geom gsh[2];
    const Vecs<T, false, false> V{Ls, nullptr, nullptr, rhs0, phi0};
    vcycle_cell_body<DIM, T, false>(ClusterSync{}, gsh, Ls, nlev, lblock, V, nu, ncoarse);
}

// Column i of the coarse-solve matrix: the ncoarse sweeps applied to e_i.
template <int DIM, typename T, bool BULK>
__global__ void __launch_bounds__(CT) k_smat_vel(Geom g, Coef<T> C, int ncoarse, T* __restrict__ st) {
    pdl_entry();
    __shared__ T phi[SMAT_MAX], rhs[SMAT_MAX];
    const int i = blockIdx.x, n = g.nvel;
    for (int t = threadIdx.x; t < n; t += CT) {
        phi[t] = T(0);
        rhs[t] = t == i ? T(1) : T(0);
    }
    __syncthreads();
    c_vel_sweeps<DIM, T, BULK>(BlockSync{}, g, C, ncoarse, phi, rhs);
    for (int t = threadIdx.x; t < n; t += CT) st[(size_t)i * n + t] = phi[t];
}

template <int DIM, typename T>
__global__ void __launch_bounds__(CT) k_smat_cell(Geom g, Coef<T> C, int ncoarse, T* __restrict__ st) {
    pdl_entry();
    __shared__ T phi[SMAT_MAX], rhs[SMAT_MAX];
    const int i = blockIdx.x, n = g.ncell;
    for (int t = threadIdx.x; t < n; t += CT) {
        phi[t] = T(0);
        rhs[t] = t == i ? T(1) : T(0);
    }
    __syncthreads();
    c_cell_sweeps<DIM, T>(BlockSync{}, g, C, ncoarse, phi, rhs);
    for (int t = threadIdx.x; t < n; t += CT) st[(size_t)i * n + t] = phi[t];
}

template <typename T>
__global__ void __launch_bounds__(CT) k_smat_apply(int n, const T* __restrict__ st, const T* __restrict__ rhs,
                                                   T* __restrict__ phi) {
    pdl_entry();
    smat_apply<T>(BlockSync{}, st, n, rhs, phi);
}

}  // namespace

template <typename T>
void launch_coarsest_matrix_vel(const Geom& g, Coef<T> C, int ncoarse, T* st, cudaStream_t s) {
    if (g.nvel > SMAT_MAX || g.nvel < 1) return;
    const bool bk = C.lam_c != nullptr;
    if (g.dim == 2)
        launch_pdl(bk ? k_smat_vel<2, T, true> : k_smat_vel<2, T, false>, dim3(g.nvel), dim3(CT), s, g, C,
                   ncoarse, st);
    else
        launch_pdl(bk ? k_smat_vel<3, T, true> : k_smat_vel<3, T, false>, dim3(g.nvel), dim3(CT), s, g, C,
                   ncoarse, st);
}

template <typename T>
void launch_coarsest_matrix_cell(const Geom& g, Coef<T> C, int ncoarse, T* st, cudaStream_t s) {
    if (g.ncell > SMAT_MAX || g.ncell < 1) return;
    if (g.dim == 2) launch_pdl(k_smat_cell<2, T>, dim3(g.ncell), dim3(CT), s, g, C, ncoarse, st);
    else launch_pdl(k_smat_cell<3, T>, dim3(g.ncell), dim3(CT), s, g, C, ncoarse, st);
}

template <typename T>
void launch_coarsest_apply(int n, const T* st, const T* rhs, T* phi, cudaStream_t s) {
    launch_pdl(k_smat_apply<T>, dim3(1), dim3(CT), s, n, st, rhs, phi);
}

template void launch_coarsest_matrix_vel<double>(const Geom&, Coef<double>, int, double*, cudaStream_t);
template void launch_coarsest_matrix_vel<float>(const Geom&, Coef<float>, int, float*, cudaStream_t);
template void launch_coarsest_matrix_cell<double>(const Geom&, Coef<double>, int, double*, cudaStream_t);
template void launch_coarsest_matrix_cell<float>(const Geom&, Coef<float>, int, float*, cudaStream_t);
template void launch_coarsest_apply<double>(int, const double*, const double*, double*, cudaStream_t);
template void launch_coarsest_apply<float>(int, const float*, const float*, float*, cudaStream_t);

// dynamic shared memory the SMEM variants may use (set on every kernel by
// prepare_coarse_kernels; the static Geom copies and layout need ~2 KB more)
constexpr size_t COARSE_SMEM_MAX = COARSE_SMEM_LIMIT;

template <typename K>
void set_smem_attr(K kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)COARSE_SMEM_MAX);
}

template <typename T>
void launch_coarse_vcycle_vel(int dim, int nsl, const CLevel<T>* L, int nlev, const T* rhs, T* phi,
                              int nu, int ncoarse, bool bulk, size_t smem, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nsl > 1 ? nsl : 1);   // a stacked batch: one block per instance
    cfg.blockDim = dim3(CT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool sm = nsl <= 1 && smem > 0 && smem <= COARSE_SMEM_MAX;
    if (!sm) cfg.dynamicSmemBytes = 0;
#define STK_CV(D, B) (sm ? k_coarse_vel<D, T, B, true> : k_coarse_vel<D, T, B, false>)
    auto kern = dim == 2 ? (bulk ? STK_CV(2, true) : STK_CV(2, false))
                         : (bulk ? STK_CV(3, true) : STK_CV(3, false));
#undef STK_CV
    cudaLaunchKernelEx(&cfg, kern, L, nlev, rhs, phi, nu, ncoarse);
}

template <typename T>
void launch_coarse_vcycle_cell(int dim, int nsl, const CLevel<T>* L, int nlev, const T* rhs, T* phi,
                               int nu, int ncoarse, size_t smem, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nsl > 1 ? nsl : 1);
    cfg.blockDim = dim3(CT);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool sm = nsl <= 1 && smem > 0 && smem <= COARSE_SMEM_MAX;
    cfg.dynamicSmemBytes = sm ? smem : 0;
    auto kern = dim == 2 ? (sm ? k_coarse_cell<2, T, true> : k_coarse_cell<2, T, false>)
                         : (sm ? k_coarse_cell<3, T, true> : k_coarse_cell<3, T, false>);
    cudaLaunchKernelEx(&cfg, kern, L, nlev, rhs, phi, nu, ncoarse);
}

template <typename T>
int grid_vcycle_blocks(const Geom& g, bool vel) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
    // about 128 points of one colour per block on the first level (FP64 work
    // is bound by the per-SM FP64 rate, so spread it), one block per SM at most
    const int pts = vel ? (g.nvel / (2 * g.dim) + 1) : (g.ncell / 2 + 1);
    int nb = (pts + (sizeof(T) == 8 ? 127 : 511)) / (sizeof(T) == 8 ? 128 : 512);
    return nb < 1 ? 1 : (nb > sms ? sms : nb);
}

template <typename K, typename... Args>
cudaError_t launch_cooperative(K kern, int nb, cudaStream_t s, unsigned* bar, Args... args) {
    cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CT, 0);
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(CT);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename T>
cudaError_t launch_grid_vcycle_vel(int dim, const Geom& g0, const CLevel<T>* L, int nlev, int lblock,
                                   const T* rhs, T* phi, int nu, int ncoarse, bool bulk, unsigned* bar,
                                   const long long* budget, int* status, cudaStream_t s) {
    const int nb = grid_vcycle_blocks<T>(g0, true);
    auto kern = dim == 2 ? (bulk ? k_grid_vel<2, T, true> : k_grid_vel<2, T, false>)
                         : (bulk ? k_grid_vel<3, T, true> : k_grid_vel<3, T, false>);
    return launch_cooperative(kern, nb, s, bar, L, nlev, lblock, rhs, phi, nu, ncoarse, bar, budget,
                              status);
}

template <typename T>
cudaError_t launch_grid_vcycle_cell(int dim, const Geom& g0, const CLevel<T>* L, int nlev, int lblock,
                                    const T* rhs, T* phi, int nu, int ncoarse, unsigned* bar,
                                    const long long* budget, int* status, cudaStream_t s) {
    const int nb = grid_vcycle_blocks<T>(g0, false);
    auto kern = dim == 2 ? k_grid_cell<2, T> : k_grid_cell<3, T>;
    return launch_cooperative(kern, nb, s, bar, L, nlev, lblock, rhs, phi, nu, ncoarse, bar, budget,
                              status);
}

template <typename T>
void launch_coarse_stacked(bool vel, int dim, int nsl, const CLevel<T>* Lall, int lstride, int nlev,
                           const T* rhs, T* phi, int nu, int ncoarse, bool bulk, size_t smem,
                           cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nsl);
    cfg.blockDim = dim3(CT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ++tl_launches;
    if (dim != 2) return;   // stacked batches are 2D
    void (*kern)(const CLevel<T>*, int, int, const T*, T*, int, int) = nullptr;
    if (vel) kern = bulk ? k_coarse_stk<2, T, true, true> : k_coarse_stk<2, T, false, true>;
    else kern = k_coarse_stk<2, T, false, false>;
    cudaLaunchKernelEx(&cfg, kern, Lall, lstride, nlev, rhs, phi, nu, ncoarse);
}

template <typename T>
void launch_faces_by_instance(const Geom& gl, int nsl, const T* src, T* dst, cudaStream_t s) {
    launch_pdl(k_faces_by_instance<T>, dim3((gl.nvel + 255) / 256, nsl), dim3(256), s, gl, nsl, src, dst);
}

template void launch_coarse_stacked<double>(bool, int, int, const CLevel<double>*, int, int, const double*,
                                            double*, int, int, bool, size_t, cudaStream_t);
template void launch_coarse_stacked<float>(bool, int, int, const CLevel<float>*, int, int, const float*,
                                           float*, int, int, bool, size_t, cudaStream_t);
template void launch_faces_by_instance<double>(const Geom&, int, const double*, double*, cudaStream_t);
template void launch_faces_by_instance<float>(const Geom&, int, const float*, float*, cudaStream_t);

// the largest cluster the device runs (16 when non-portable sizes are
// allowed and fit one GPC, else 8); set by prepare_coarse_kernels
static int g_cluster_max = 8;

template <typename K>
int max_cluster(K kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int c = 16; c >= 2; c /= 2) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(CT);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n >= 1) return c;
        cudaGetLastError();
    }
    return 1;
}

template <typename K, typename... Args>
cudaError_t launch_cluster(K kern, int nb, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(CT);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = nb;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename T>
int cluster_vcycle_blocks(const Geom& g0, bool vel) {
    const int nb = grid_vcycle_blocks<T>(g0, vel);
    return nb < g_cluster_max ? nb : g_cluster_max;
}

template <typename T>
cudaError_t launch_cluster_vcycle_vel(int dim, const Geom& g0, const CLevel<T>* L, int nlev, int lblock,
                                      const T* rhs, T* phi, int nu, int ncoarse, bool bulk, cudaStream_t s) {
    const int nb = cluster_vcycle_blocks<T>(g0, true);
    auto kern = dim == 2 ? (bulk ? k_cluster_vel<2, T, true> : k_cluster_vel<2, T, false>)
                         : (bulk ? k_cluster_vel<3, T, true> : k_cluster_vel<3, T, false>);
    ++tl_launches;
    return launch_cluster(kern, nb, s, L, nlev, lblock, rhs, phi, nu, ncoarse);
}

template <typename T>
cudaError_t launch_cluster_vcycle_cell(int dim, const Geom& g0, const CLevel<T>* L, int nlev, int lblock,
                                       const T* rhs, T* phi, int nu, int ncoarse, cudaStream_t s) {
    const int nb = cluster_vcycle_blocks<T>(g0, false);
    auto kern = dim == 2 ? k_cluster_cell<2, T> : k_cluster_cell<3, T>;
    ++tl_launches;
    return launch_cluster(kern, nb, s, L, nlev, lblock, rhs, phi, nu, ncoarse);
}

template cudaError_t launch_cluster_vcycle_vel<double>(int, const Geom&, const CLevel<double>*, int, int,
                                                       const double*, double*, int, int, bool, cudaStream_t);
template cudaError_t launch_cluster_vcycle_vel<float>(int, const Geom&, const CLevel<float>*, int, int,
                                                      const float*, float*, int, int, bool, cudaStream_t);
template cudaError_t launch_cluster_vcycle_cell<double>(int, const Geom&, const CLevel<double>*, int, int,
                                                        const double*, double*, int, int, cudaStream_t);
template cudaError_t launch_cluster_vcycle_cell<float>(int, const Geom&, const CLevel<float>*, int, int,
                                                       const float*, float*, int, int, cudaStream_t);

template cudaError_t launch_grid_vcycle_vel<double>(int, const Geom&, const CLevel<double>*, int, int,
                                                    const double*, double*, int, int, bool, unsigned*,
                                                    const long long*, int*, cudaStream_t);
template cudaError_t launch_grid_vcycle_vel<float>(int, const Geom&, const CLevel<float>*, int, int,
                                                   const float*, float*, int, int, bool, unsigned*,
                                                   const long long*, int*, cudaStream_t);
template cudaError_t launch_grid_vcycle_cell<double>(int, const Geom&, const CLevel<double>*, int, int,
                                                     const double*, double*, int, int, unsigned*,
                                                     const long long*, int*, cudaStream_t);
template cudaError_t launch_grid_vcycle_cell<float>(int, const Geom&, const CLevel<float>*, int, int,
                                                    const float*, float*, int, int, unsigned*,
                                                    const long long*, int*, cudaStream_t);

void prepare_coarse_kernels() {
    static bool clusters_done = false;
    if (!clusters_done) {   // every cluster kernel uses 1024 threads and the same static memory
        clusters_done = true;
        int c = max_cluster(k_cluster_vel<3, double, false>);
        const auto all = {k_cluster_vel<2, double, false>, k_cluster_vel<2, double, true>,
                          k_cluster_vel<3, double, false>, k_cluster_vel<3, double, true>};
        for (auto k : all) cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        const auto allf = {k_cluster_vel<2, float, false>, k_cluster_vel<2, float, true>,
                           k_cluster_vel<3, float, false>, k_cluster_vel<3, float, true>};
        for (auto k : allf) cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        const auto allc = {k_cluster_cell<2, double>, k_cluster_cell<3, double>};
        for (auto k : allc) cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        const auto allcf = {k_cluster_cell<2, float>, k_cluster_cell<3, float>};
        for (auto k : allcf) cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        for (auto k : allf) c = std::min(c, max_cluster(k));
        for (auto k : all) c = std::min(c, max_cluster(k));
        for (auto k : allc) c = std::min(c, max_cluster(k));
        for (auto k : allcf) c = std::min(c, max_cluster(k));
        g_cluster_max = c;
        cudaGetLastError();
    }
    set_smem_attr(k_coarse_vel<2, double, false, true>);
    set_smem_attr(k_coarse_vel<3, double, false, true>);
    set_smem_attr(k_coarse_vel<2, double, true, true>);
    set_smem_attr(k_coarse_vel<3, double, true, true>);
    set_smem_attr(k_coarse_vel<2, float, false, true>);
    set_smem_attr(k_coarse_vel<3, float, false, true>);
    set_smem_attr(k_coarse_vel<2, float, true, true>);
    set_smem_attr(k_coarse_vel<3, float, true, true>);
    set_smem_attr(k_coarse_stk<2, double, false, true>);
    set_smem_attr(k_coarse_stk<2, double, true, true>);
    set_smem_attr(k_coarse_stk<2, double, false, false>);
    set_smem_attr(k_coarse_stk<2, float, false, true>);
    set_smem_attr(k_coarse_stk<2, float, true, true>);
    set_smem_attr(k_coarse_stk<2, float, false, false>);
    set_smem_attr(k_coarse_cell<2, double, true>);
    set_smem_attr(k_coarse_cell<3, double, true>);
    set_smem_attr(k_coarse_cell<2, float, true>);
    set_smem_attr(k_coarse_cell<3, float, true>);
}

template void launch_coarse_vcycle_vel<double>(int, int, const CLevel<double>*, int, const double*,
                                               double*, int, int, bool, size_t, cudaStream_t);
template void launch_coarse_vcycle_vel<float>(int, int, const CLevel<float>*, int, const float*, float*,
                                              int, int, bool, size_t, cudaStream_t);
template void launch_coarse_vcycle_cell<double>(int, int, const CLevel<double>*, int, const double*,
                                                double*, int, int, size_t, cudaStream_t);
template void launch_coarse_vcycle_cell<float>(int, int, const CLevel<float>*, int, const float*,
                                               float*, int, int, size_t, cudaStream_t);

STK_OOB_READER(coarse)

}  // namespace stk
