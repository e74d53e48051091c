// Both colours of one Gauss-Seidel sweep in one launch (App. C smoother).
//
// The per-colour kernels (kernels.cu) read every input array once per colour
// and the second colour waits for a grid-wide launch boundary.  Here a block
// owns a tile of one face (or cell) array and does both colours itself:
//
//   1. the red points ((i + j + k) even) of the tile and of a one-point halo
//      around it are computed from the input values into shared memory (the
//      halo points belong to neighbouring tiles and are recomputed, with the
//      same arithmetic, from the same inputs);
//   2. the black points of the tile are computed from those red values.
//
// The sweep is out of place: values are read from `src` and written to
// `dst`, so no block ever reads a value that another block of the same
// launch writes.  For the velocity, a sweep over components x, y(, z) reads
// the components already swept from `dst` and the others from `src`; after
// a whole sweep every component lives in `dst`, and the caller swaps the two
// buffers.  The results equal those of the two per-colour launches: the
// same per-point functions (stencil.cuh) with the same operands.
#include "stencil.cuh"

namespace stk {
namespace {

using namespace st;

// In-range coordinate of the (unwrapped) position u along axis d of an
// array with extent e, or -1 if there is none: periodic axes wrap once,
// other axes end at the array.
__device__ __forceinline__ int halo_coord(const Geom& g, int d, int u, int e) {
    if (g.per[d]) return (u < -1 || u > e) ? -1 : wrapm(u, e);
    return (u < 0 || u >= e) ? -1 : u;
}
// Shared-memory slot of in-range coordinate c of a neighbour of a tile point,
// for a haloed tile that starts at o (tile origin - 1) and is W wide; a
// neighbour across a periodic seam is found one period away.
__device__ __forceinline__ int slot(int c, int o, int W, int e) {
    int l = c - o;
    if (l < 0) l += e;
    else if (l >= W) l -= e;
    return l;
}

// Velocity component A.  Tile: 2 TXC faces along x (TXC of each colour),
// TY along y, TZ along z (3D); one thread per black point.
template <int DIM, int A, typename T, int TXC, int TY, int TZ, bool BULK>
__global__ void __launch_bounds__(TXC * TY * TZ)
k_vel_gs_pair(Geom g, Coef<T> C, const T* src, T* dst, const T* __restrict__ rhs) {
    pdl_entry();
    constexpr int NT = TXC * TY * TZ;
    constexpr int WX = 2 * TXC + 2, WY = TY + 2, WZ = DIM == 3 ? TZ + 2 : 1;
    __shared__ T R[WZ][WY][WX];
    const int e0 = g.fe[A][0], e1 = g.fe[A][1], e2 = g.fe[A][2];
    const int ox = blockIdx.x * 2 * TXC - 1, oy = blockIdx.y * TY - 1;
    const int oz = DIM == 3 ? int(blockIdx.z) * TZ - 1 : 0;
    const int sl = DIM == 3 ? 0 : int(blockIdx.z);   // 2D: the instance of a stacked batch
    // components swept before A in this sweep are in dst, the others in src
    auto pb = [&](int B, int i) { return T((B < A ? dst : src)[i]); };

    // 1. red points of the haloed tile, from the input values
    {
        auto aidx = [&](const int* r) { return fidx(g, A, r); };
        auto ga = [&](int i) { return T(src[i]); };
        for (int t = threadIdx.x; t < (TXC + 1) * WY * WZ; t += NT) {
            const int xr = t % (TXC + 1);
            const int rr = t / (TXC + 1);
            const int ly = rr % WY;
            const int lz = DIM == 3 ? rr / WY : 0;
            const int uy = oy + ly, uz = oz + lz;
            const int lx = 2 * xr + ((ox + uy + uz) & 1);   // ox + lx + uy + uz even
            const int ux = ox + lx;
            R[lz][ly][lx ^ 1] = T(0);   // black slot: never read, kept finite
            int q[3];
            q[0] = halo_coord(g, 0, ux, e0);
            q[1] = halo_coord(g, 1, uy, e1);
            q[2] = DIM == 3 ? halo_coord(g, 2, uz, e2) : sl;
            if (q[0] < 0 || q[1] < 0 || q[2] < 0) {
                R[lz][ly][lx] = T(0);
                continue;
            }
            T v = T(0);
            if (!wall_face(g, A, q)) {
                T dsum;
                const T N = visc_offdiag_acc<DIM, A, T, false, BULK>(g, C, q, aidx, ga, pb, dsum);
                const int f = fidx(g, A, q);
                v = vel_gs_value<T>(g, C, f, N, rhs);
                const bool inner = lx >= 1 && lx <= 2 * TXC && ux < e0 && ly >= 1 && ly <= TY &&
                                   uy < e1 && (DIM == 2 || (lz >= 1 && lz <= TZ && uz < e2));
                if (inner) dst[f] = v;
            }
            R[lz][ly][lx] = v;   // wall faces hold 0
        }
    }
    __syncthreads();

    // 2. black points of the tile, from the red values in shared memory
    const int xb = threadIdx.x % TXC;
    const int ly = 1 + (threadIdx.x / TXC) % TY;
    const int lz = DIM == 3 ? 1 + int(threadIdx.x) / (TXC * TY) : 0;
    const int uy = oy + ly, uz = oz + lz;
    const int lx = 1 + 2 * xb + ((ox + uy + uz) & 1);   // ox + lx + uy + uz odd
    const int ux = ox + lx;
    if (ux >= e0 || uy >= e1 || (DIM == 3 && uz >= e2)) return;
    const int q[3] = {ux, uy, DIM == 3 ? uz : sl};
    if (wall_face(g, A, q)) return;
    auto aidx = [&](const int* r) {
        const int sx = slot(r[0], ox, WX, e0);
        const int sy = slot(r[1], oy, WY, e1);
        const int sz = DIM == 3 ? slot(r[2], oz, WZ, e2) : 0;
        return STK_IDX((sz * WY + sy) * WX + sx, WZ * WY * WX, 4);
    };
    const T* Rf = &R[0][0][0];
    auto ga = [&](int i) { return Rf[i]; };
    T dsum;
    const T N = visc_offdiag_acc<DIM, A, T, false, BULK>(g, C, q, aidx, ga, pb, dsum);
    const int f = fidx(g, A, q);
    dst[f] = vel_gs_value<T>(g, C, f, N, rhs);
}

// Cells.  Tile: 2 TXC cells along x, TY along y, TZ along z (3D).
template <int DIM, typename T, int TXC, int TY, int TZ>
__global__ void __launch_bounds__(TXC * TY * TZ)
k_cell_gs_pair(Geom g, Coef<T> C, const T* src, T* dst, const T* __restrict__ rhs) {
    pdl_entry();
    constexpr int NT = TXC * TY * TZ;
    constexpr int WX = 2 * TXC + 2, WY = TY + 2, WZ = DIM == 3 ? TZ + 2 : 1;
    __shared__ T R[WZ][WY][WX];
    const int e0 = g.n[0], e1 = g.n[1], e2 = g.n[2];
    const int ox = blockIdx.x * 2 * TXC - 1, oy = blockIdx.y * TY - 1;
    const int oz = DIM == 3 ? int(blockIdx.z) * TZ - 1 : 0;
    const int sl = DIM == 3 ? 0 : int(blockIdx.z);   // 2D: the instance of a stacked batch
    {
        auto pc = [&](const int* r) { return T(src[cidx(g, r)]); };
        for (int t = threadIdx.x; t < (TXC + 1) * WY * WZ; t += NT) {
            const int xr = t % (TXC + 1);
            const int rr = t / (TXC + 1);
            const int ly = rr % WY;
            const int lz = DIM == 3 ? rr / WY : 0;
            const int uy = oy + ly, uz = oz + lz;
            const int lx = 2 * xr + ((ox + uy + uz) & 1);
            const int ux = ox + lx;
            // the black slot is read with weight 0 by a point next to a wall
            // (its clamped neighbour is itself), so it must hold a finite value
            R[lz][ly][lx ^ 1] = T(0);
            int q[3];
            q[0] = halo_coord(g, 0, ux, e0);
            q[1] = halo_coord(g, 1, uy, e1);
            q[2] = DIM == 3 ? halo_coord(g, 2, uz, e2) : sl;
            if (q[0] < 0 || q[1] < 0 || q[2] < 0) {
                R[lz][ly][lx] = T(0);
                continue;
            }
            const T v = cell_gs_value<DIM, T>(g, C, q, pc, rhs);
            const bool inner = lx >= 1 && lx <= 2 * TXC && ux < e0 && ly >= 1 && ly <= TY &&
                               uy < e1 && (DIM == 2 || (lz >= 1 && lz <= TZ && uz < e2));
            if (inner) dst[cidx(g, q)] = v;
            R[lz][ly][lx] = v;
        }
    }
    __syncthreads();
    const int xb = threadIdx.x % TXC;
    const int ly = 1 + (threadIdx.x / TXC) % TY;
    const int lz = DIM == 3 ? 1 + int(threadIdx.x) / (TXC * TY) : 0;
    const int uy = oy + ly, uz = oz + lz;
    const int lx = 1 + 2 * xb + ((ox + uy + uz) & 1);
    const int ux = ox + lx;
    if (ux >= e0 || uy >= e1 || (DIM == 3 && uz >= e2)) return;
    const int q[3] = {ux, uy, DIM == 3 ? uz : sl};
    auto pc = [&](const int* r) {
        const int sx = slot(r[0], ox, WX, e0);
        const int sy = slot(r[1], oy, WY, e1);
        const int sz = DIM == 3 ? slot(r[2], oz, WZ, e2) : 0;
        return (&R[0][0][0])[STK_IDX((sz * WY + sy) * WX + sx, WZ * WY * WX, 4)];
    };
    dst[cidx(g, q)] = cell_gs_value<DIM, T>(g, C, q, pc, rhs);
}

// 3D: z-marching variant.  A block owns a column of 2 TXC x TY faces
// (cells) in x, y and marches through KZ planes along z.  Stepping to plane
// kb + 1 it computes the red points of that plane on the haloed tile (from
// the input values, into a ring of three shared-memory planes), then the
// black points of plane kb, whose red neighbours in planes kb - 1, kb and
// kb + 1 are all in the ring.  Every input plane is read about once per
// sweep and component (instead of once per colour), the halo recomputation
// is one ring of points in x, y and two planes per column.  Out of place and
// with the same per-point arithmetic, as above.

// Ring slot of the plane kb + d (d = -1, 0, 1) holding the (wrapped) plane
// coordinate z: the plane offset is recovered from z itself, so neighbours
// across a periodic seam are found.
__device__ __forceinline__ int ring_slot(const Geom& g, int z, int kb, int e2) {
    const int up = g.per[2] ? wrapm(kb + 1, e2) : kb + 1;
    const int d = z == kb ? 0 : (z == up ? 1 : -1);
    return (kb + d + 3) % 3;
}
// wrapped coordinate of plane kr (-1 <= kr <= e2), or -1 if there is none
__device__ __forceinline__ int plane_coord(const Geom& g, int kr, int e2) {
    if (g.per[2]) return wrapm(kr, e2);
    return (kr < 0 || kr >= e2) ? -1 : kr;
}

template <int A, typename T, int TXC, int TY, int KZ, bool BULK>
__global__ void __launch_bounds__(TXC * TY)
k_vel_gs_zpair(Geom g, Coef<T> C, const T* src, T* dst, const T* __restrict__ rhs) {
    pdl_entry();
    constexpr int NT = TXC * TY;
    constexpr int WX = 2 * TXC + 2, WY = TY + 2;
    __shared__ T R[3][WY][WX];
    const int e0 = g.fe[A][0], e1 = g.fe[A][1], e2 = g.fe[A][2];
    const int ox = blockIdx.x * 2 * TXC - 1, oy = blockIdx.y * TY - 1;
    const int k0 = blockIdx.z * KZ;
    const int k1 = min(k0 + KZ, e2);   // this block's planes [k0, k1)
    auto pb = [&](int B, int i) { return T((B < A ? dst : src)[i]); };
    auto gidx = [&](const int* r) { return fidx(g, A, r); };
    auto gsrc = [&](int i) { return T(src[i]); };

    auto red_plane = [&](int kr) {
        const int sz = (kr + 3) % 3;
        const int kw = plane_coord(g, kr, e2);
        for (int t = threadIdx.x; t < (TXC + 1) * WY; t += NT) {
            const int xr = t % (TXC + 1);
            const int ly = t / (TXC + 1);
            const int uy = oy + ly;
            const int lx = 2 * xr + ((ox + uy + kr) & 1);   // ox + lx + uy + kr even
            const int ux = ox + lx;
            R[sz][ly][lx ^ 1] = T(0);   // black slot: never read, kept finite
            int q[3];
            q[0] = halo_coord(g, 0, ux, e0);
            q[1] = halo_coord(g, 1, uy, e1);
            q[2] = kw;
            if (q[0] < 0 || q[1] < 0 || q[2] < 0) {
                R[sz][ly][lx] = T(0);
                continue;
            }
            T v = T(0);
            if (!wall_face(g, A, q)) {
                T dsum;
                const T N = visc_offdiag_acc<3, A, T, false, BULK>(g, C, q, gidx, gsrc, pb, dsum);
                const int f = fidx(g, A, q);
                v = vel_gs_value<T>(g, C, f, N, rhs);
                const bool inner = lx >= 1 && lx <= 2 * TXC && ux < e0 && ly >= 1 && ly <= TY &&
                                   uy < e1 && kr >= k0 && kr < k1;
                if (inner) dst[f] = v;
            }
            R[sz][ly][lx] = v;   // wall faces hold 0
        }
    };
    const T* Rf = &R[0][0][0];
    auto black_plane = [&](int kb) {
        const int xb = threadIdx.x % TXC;
        const int ly = 1 + threadIdx.x / TXC;
        const int uy = oy + ly;
        const int lx = 1 + 2 * xb + ((ox + uy + kb) & 1);   // ox + lx + uy + kb odd
        const int ux = ox + lx;
        if (ux >= e0 || uy >= e1) return;
        const int q[3] = {ux, uy, kb};
        if (wall_face(g, A, q)) return;
        auto aidx = [&](const int* r) {
            const int sx = slot(r[0], ox, WX, e0);
            const int sy = slot(r[1], oy, WY, e1);
            return STK_IDX((ring_slot(g, r[2], kb, e2) * WY + sy) * WX + sx, 3 * WY * WX, 4);
        };
        auto ga = [&](int i) { return Rf[i]; };
        T dsum;
        const T N = visc_offdiag_acc<3, A, T, false, BULK>(g, C, q, aidx, ga, pb, dsum);
        const int f = fidx(g, A, q);
        dst[f] = vel_gs_value<T>(g, C, f, N, rhs);
    };
    red_plane(k0 - 1);
    red_plane(k0);
    for (int kb = k0; kb < k1; ++kb) {
        red_plane(kb + 1);
        __syncthreads();
        black_plane(kb);
        __syncthreads();
    }
}

template <typename T, int TXC, int TY, int KZ>
__global__ void __launch_bounds__(TXC * TY)
k_cell_gs_zpair(Geom g, Coef<T> C, const T* src, T* dst, const T* __restrict__ rhs) {
    pdl_entry();
    constexpr int NT = TXC * TY;
    constexpr int WX = 2 * TXC + 2, WY = TY + 2;
    __shared__ T R[3][WY][WX];
    const int e0 = g.n[0], e1 = g.n[1], e2 = g.n[2];
    const int ox = blockIdx.x * 2 * TXC - 1, oy = blockIdx.y * TY - 1;
    const int k0 = blockIdx.z * KZ;
    const int k1 = min(k0 + KZ, e2);
    auto red_plane = [&](int kr) {
        const int sz = (kr + 3) % 3;
        const int kw = plane_coord(g, kr, e2);
        auto pc = [&](const int* r) { return T(src[cidx(g, r)]); };
        for (int t = threadIdx.x; t < (TXC + 1) * WY; t += NT) {
            const int xr = t % (TXC + 1);
            const int ly = t / (TXC + 1);
            const int uy = oy + ly;
            const int lx = 2 * xr + ((ox + uy + kr) & 1);
            const int ux = ox + lx;
            // the black slot is read with weight 0 by a point next to a wall
            // (its clamped neighbour is itself), so it must hold a finite value
            R[sz][ly][lx ^ 1] = T(0);
            int q[3];
            q[0] = halo_coord(g, 0, ux, e0);
            q[1] = halo_coord(g, 1, uy, e1);
            q[2] = kw;
            if (q[0] < 0 || q[1] < 0 || q[2] < 0) {
                R[sz][ly][lx] = T(0);
                continue;
            }
            const T v = cell_gs_value<3, T>(g, C, q, pc, rhs);
            const bool inner = lx >= 1 && lx <= 2 * TXC && ux < e0 && ly >= 1 && ly <= TY &&
                               uy < e1 && kr >= k0 && kr < k1;
            if (inner) dst[cidx(g, q)] = v;
            R[sz][ly][lx] = v;
        }
    };
    auto black_plane = [&](int kb) {
        const int xb = threadIdx.x % TXC;
        const int ly = 1 + threadIdx.x / TXC;
        const int uy = oy + ly;
        const int lx = 1 + 2 * xb + ((ox + uy + kb) & 1);
        const int ux = ox + lx;
        if (ux >= e0 || uy >= e1) return;
        const int q[3] = {ux, uy, kb};
        auto pc = [&](const int* r) {
            const int sx = slot(r[0], ox, WX, e0);
            const int sy = slot(r[1], oy, WY, e1);
            return (&R[0][0][0])[STK_IDX((ring_slot(g, r[2], kb, e2) * WY + sy) * WX + sx, 3 * WY * WX, 4)];
        };
        dst[cidx(g, q)] = cell_gs_value<3, T>(g, C, q, pc, rhs);
    };
    red_plane(k0 - 1);
    red_plane(k0);
    for (int kb = k0; kb < k1; ++kb) {
        red_plane(kb + 1);
        __syncthreads();
        black_plane(kb);
        __syncthreads();
    }
}

// tile shapes: 2D 32 x 16 (256 threads; grid z = the instances of a stacked
// batch); 3D z-march columns of 64 x 8 faces (256 threads) through 16 planes
constexpr int P2X = 16, P2Y = 16;
constexpr int Z3X = 32, Z3Y = 8, Z3K = 16;

inline dim3 pair_grid(int dim, int e0, int e1, int e2) {
    if (dim == 2) return dim3((e0 + 2 * P2X - 1) / (2 * P2X), (e1 + P2Y - 1) / P2Y, e2);
    return dim3((e0 + 2 * Z3X - 1) / (2 * Z3X), (e1 + Z3Y - 1) / Z3Y, (e2 + Z3K - 1) / Z3K);
}

}  // namespace

template <typename T>
void launch_vel_gs_pair(const Geom& g, Coef<T> C, int comp, const T* src, T* dst, const T* rhs,
                        cudaStream_t s) {
    const dim3 gr = pair_grid(g.dim, g.fe[comp][0], g.fe[comp][1], g.fe[comp][2]);
    const bool bk = C.lam_c != nullptr;
#define STK_P2(A) (bk ? k_vel_gs_pair<2, A, T, P2X, P2Y, 1, true> : k_vel_gs_pair<2, A, T, P2X, P2Y, 1, false>)
#define STK_P3(A) (bk ? k_vel_gs_zpair<A, T, Z3X, Z3Y, Z3K, true> : k_vel_gs_zpair<A, T, Z3X, Z3Y, Z3K, false>)
    if (g.dim == 2) {
        const dim3 bl(P2X * P2Y);
        if (comp == 0) launch_pdl(STK_P2(0), gr, bl, s, g, C, src, dst, rhs);
        else launch_pdl(STK_P2(1), gr, bl, s, g, C, src, dst, rhs);
    } else {
        const dim3 bl(Z3X * Z3Y);
        if (comp == 0) launch_pdl(STK_P3(0), gr, bl, s, g, C, src, dst, rhs);
        else if (comp == 1) launch_pdl(STK_P3(1), gr, bl, s, g, C, src, dst, rhs);
        else launch_pdl(STK_P3(2), gr, bl, s, g, C, src, dst, rhs);
    }
#undef STK_P2
#undef STK_P3
}

template <typename T>
void launch_cell_gs_pair(const Geom& g, Coef<T> C, const T* src, T* dst, const T* rhs,
                         cudaStream_t s) {
    const dim3 gr = pair_grid(g.dim, g.n[0], g.n[1], g.n[2]);
    if (g.dim == 2) launch_pdl(k_cell_gs_pair<2, T, P2X, P2Y, 1>, gr, dim3(P2X * P2Y), s, g, C, src, dst, rhs);
    else launch_pdl(k_cell_gs_zpair<T, Z3X, Z3Y, Z3K>, gr, dim3(Z3X * Z3Y), s, g, C, src, dst, rhs);
}

template void launch_vel_gs_pair<double>(const Geom&, Coef<double>, int, const double*, double*,
                                         const double*, cudaStream_t);
template void launch_vel_gs_pair<float>(const Geom&, Coef<float>, int, const float*, float*,
                                        const float*, cudaStream_t);
template void launch_cell_gs_pair<double>(const Geom&, Coef<double>, const double*, double*,
                                          const double*, cudaStream_t);
template void launch_cell_gs_pair<float>(const Geom&, Coef<float>, const float*, float*,
                                         const float*, cudaStream_t);

STK_OOB_READER(pair)

}  // namespace stk
