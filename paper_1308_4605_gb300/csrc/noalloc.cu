// stk_pressure_vcycle_noalloc: the pressure V-cycle of stk_pressure_vcycle
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: an application whose device memory is
// wholly owned by another allocator (a framework that reserves the GPU's
// memory pool up front, so a stray cudaMalloc fails or fragments that pool),
// or a latency-critical loop in which the implicit synchronisation of
// cudaMalloc/cudaFree is not acceptable.  They cannot create an stk_handle
// (stk_create allocates its workspace), so this entry point takes the
// density and the right-hand side directly and keeps its whole multigrid
// workspace (face coefficients, inverse diagonals, coarse work vectors) in one
// file-scope device array of fixed size.  Every GPU that loads this library
// holds that array until the process exits.
//
// It runs the same V-cycle as stk_pressure_vcycle on a handle whose
// coefficients were set with the same rho, equal to it up to rounding: the
// smoothing, residual and transfer kernels are those of kernels.cu, while the
// coefficient setup (k_na_fine_beta, k_na_coarse_beta, k_na_invdiag) is a
// local copy of the same formulas that sums the diagonal in its own order, and
// the coarsest level is swept 8 times (the handle applies those sweeps as a
// precomputed matrix).  A change to the face coefficients or their coarsening
// in kernels.cu must be mirrored here.
//
// With CUDA's lazy module loading (the default since CUDA 12.2) the scratch
// array and the code of the kernels used here are placed in device memory
// when the first call on a device runs, not when the library is loaded: a
// caller whose allocator is about to reserve the device memory makes one
// warm-up call first.
#include "internal.cuh"
#include "../../include/stokes.h"

#include <cmath>
#include <mutex>

namespace {

// 2,097,152 doubles = 16 MiB: enough for 2D grids up to 512^2 and 3D grids
// up to 64^3 (the workspace is about 6 doubles per cell).
constexpr long long kScratchWords = 2LL << 20;

}  // namespace

static __device__ __align__(256) double g_stk_noalloc_scratch[kScratchWords];

namespace {

using stk::Geom;

std::mutex g_setup_mutex;
constexpr int kMaxDevices = 256;
double* g_scratch_addr[kMaxDevices] = {};

__device__ __forceinline__ int na_wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
__device__ __forceinline__ int na_fidx(const Geom& g, int a, const int q[3]) {
    return g.foff[a] + (q[2] * g.fe[a][1] + q[1]) * g.fe[a][0] + q[0];
}
__device__ __forceinline__ int na_cidx(const Geom& g, const int q[3]) {
    return (q[2] * g.n[1] + q[1]) * g.n[0] + q[0];
}
__device__ __forceinline__ void na_decode(int t, const int e[3], int q[3]) {
    q[0] = t % e[0];
    int r = t / e[0];
    q[1] = r % e[1];
    q[2] = r / e[1];
}

// beta = 1 / rho_f on unknown faces, rho_f the mean of the two adjacent cells
// (Sec. 3.1); 0 on wall faces.
__global__ void k_na_fine_beta(Geom g, const double* __restrict__ rho, double* beta) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.nvel) return;
    int a = 0;
    while (a + 1 < g.dim && t >= g.foff[a + 1]) ++a;
    int q[3];
    na_decode(t - g.foff[a], g.fe[a], q);
    if (!g.per[a] && (q[a] == 0 || q[a] == g.n[a])) {
        beta[t] = 0.0;
        return;
    }
    int qm[3] = {q[0], q[1], q[2]};
    qm[a] = g.per[a] ? na_wrap(q[a] - 1, g.n[a]) : q[a] - 1;
    double rf = 0.5 * (rho[na_cidx(g, q)] + rho[na_cidx(g, qm)]);
    beta[t] = 1.0 / rf;
}

// coarse face beta = mean of the overlying fine faces (App. C)
__global__ void k_na_coarse_beta(Geom gf, Geom gc, const double* __restrict__ bf, double* bc) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= gc.nvel) return;
    int a = 0;
    while (a + 1 < gc.dim && t >= gc.foff[a + 1]) ++a;
    int Q[3];
    na_decode(t - gc.foff[a], gc.fe[a], Q);
    int tb[2], nt = 0;
    for (int b = 0; b < gc.dim; ++b)
        if (b != a) tb[nt++] = b;
    double sb = 0.0;
    int cnt = 0;
    for (int m = 0; m < (1 << nt); ++m) {
        int q[3] = {2 * Q[0], 2 * Q[1], gc.dim == 3 ? 2 * Q[2] : 0};
        for (int k = 0; k < nt; ++k) q[tb[k]] += (m >> k) & 1;
        sb += bf[na_fidx(gf, a, q)];
        ++cnt;
    }
    bc[t] = sb / cnt;
}

// inverse diagonal of L_rho = D beta G
__global__ void k_na_invdiag(Geom g, const double* __restrict__ beta, double* invd) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ncell) return;
    int q[3];
    na_decode(t, g.n, q);
    double d = 0.0;
    for (int a = 0; a < g.dim; ++a) {
        int fh[3] = {q[0], q[1], q[2]};
        fh[a] = g.per[a] ? na_wrap(q[a] + 1, g.n[a]) : q[a] + 1;
        d -= g.ih2 * (beta[na_fidx(g, a, fh)] + beta[na_fidx(g, a, q)]);
    }
    invd[t] = d != 0.0 ? 1.0 / d : 0.0;
}

Geom na_geom(int dim, const int n[3], double hh, const int bc[6]) {
    Geom g{};
    g.dim = dim;
    g.nsl = 1;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = a < dim ? n[a] : 1;
        g.per[a] = a < dim ? (bc[2 * a] == STK_PERIODIC) : 1;
        g.bclo[a] = a < dim ? bc[2 * a] : STK_PERIODIC;
        g.bchi[a] = a < dim ? bc[2 * a + 1] : STK_PERIODIC;
    }
    int off = 0;
    for (int a = 0; a < 3; ++a) {
        for (int c = 0; c < 3; ++c) g.fe[a][c] = g.n[c] + ((c == a && !g.per[a]) ? 1 : 0);
        g.fsize[a] = a < dim ? g.fe[a][0] * g.fe[a][1] * g.fe[a][2] : 0;
        g.foff[a] = off;
        off += g.fsize[a];
    }
    g.nvel = off;
    g.ncell = g.n[0] * g.n[1] * g.n[2];
    g.h = hh;
    g.ih = 1.0 / hh;
    g.ih2 = 1.0 / (hh * hh);
    stk::finish_geom(g);
    return g;
}

struct NaLevel {
    Geom g;
    stk::Coef<double> C;   // beta and invd_p used
    double *phi, *rhs, *res;
};

constexpr int kMaxLevels = 16;

void na_vcycle(NaLevel* L, int nlev, int l, const double* rhs, double* phi, cudaStream_t s) {
    const int nu = 2, ncoarse = 8;   // App. C / Sec. 4.1.1, as stk_pressure_vcycle
    const NaLevel& Lv = L[l];
    cudaMemsetAsync(phi, 0, sizeof(double) * Lv.g.ncell, s);
    auto sweeps = [&](int k) {
        for (int it = 0; it < k; ++it)
            for (int par = 0; par < 2; ++par)
                stk::launch_cell_gs_colour<double>(Lv.g, Lv.C, par, phi, rhs, s);
    };
    if (l + 1 == nlev) {
        sweeps(ncoarse);
        return;
    }
    sweeps(nu);
    stk::launch_cell_residual<double>(Lv.g, Lv.C, phi, rhs, Lv.res, s, true);
    stk::launch_cell_restrict<double>(Lv.g, Lv.res, L[l + 1].g, L[l + 1].rhs, s);
    na_vcycle(L, nlev, l + 1, L[l + 1].rhs, L[l + 1].phi, s);
    stk::launch_cell_prolong_add<double>(L[l + 1].g, L[l + 1].phi, Lv.g, phi, s);
    sweeps(nu);
}

bool na_pow2(int v) { return v >= 2 && (v & (v - 1)) == 0; }

}  // namespace

extern "C" int stk_pressure_vcycle_noalloc(int dim, const int* n, double h, const int* bc,
                                           const double* rho, const double* r_p, double* x_p,
                                           void* stream) {
    if (dim != 2 && dim != 3) return STK_ERR_ARG;
    // an error left pending by the caller's earlier work is reported as
    // STK_ERR_CUDA and left in place (peeked, not cleared), so that the
    // final check below sees only this call's launches
    if (cudaPeekAtLastError() != cudaSuccess) return STK_ERR_CUDA;
    if (!n || !bc || !rho || !r_p || !x_p) return STK_ERR_ARG;
    if (!(h > 0.0) || !std::isfinite(h)) return STK_ERR_ARG;
    int nn[3] = {1, 1, 1}, bb[6] = {0, 0, 0, 0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        if (!na_pow2(n[a])) return STK_ERR_SIZE;
        nn[a] = n[a];
        bb[2 * a] = bc[2 * a];
        bb[2 * a + 1] = bc[2 * a + 1];
        for (int sd = 0; sd < 2; ++sd)
            if (bb[2 * a + sd] < 0 || bb[2 * a + sd] > 2) return STK_ERR_ARG;
        if ((bb[2 * a] == STK_PERIODIC) != (bb[2 * a + 1] == STK_PERIODIC)) return STK_ERR_ARG;
    }
    if ((long long)nn[0] * nn[1] * nn[2] > kScratchWords) return STK_ERR_SIZE;
    // hierarchy and workspace size (checked before any device work)
    NaLevel L[kMaxLevels];
    int nlev = 0;
    long long words = 0;
    {
        int cur[3] = {nn[0], nn[1], nn[2]};
        double hl = h;
        while (true) {
            if (nlev == kMaxLevels) return STK_ERR_SIZE;
            Geom g = na_geom(dim, cur, hl, bb);
            L[nlev].g = g;
            // beta, invd, res above the coarsest level, and phi, rhs below
            // the finest level; every array starts on a 256-byte boundary
            // (as carved below)
            auto rounded = [](long long c) { return (c + 31) & ~31LL; };
            int mn = cur[0];
            for (int a = 1; a < dim; ++a) mn = cur[a] < mn ? cur[a] : mn;
            const bool coarsest = mn <= 2;
            words += rounded(g.nvel) + rounded(g.ncell) + (coarsest ? 0 : rounded(g.ncell)) +
                     (nlev > 0 ? 2 * rounded(g.ncell) : 0);
            ++nlev;
            if (coarsest) break;
            for (int a = 0; a < dim; ++a) cur[a] /= 2;
            hl *= 2.0;
        }
    }
    if (words > kScratchWords) return STK_ERR_SIZE;

    // once per device: the device address of the scratch array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return STK_ERR_CUDA;
    double* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_stk_noalloc_scratch) != cudaSuccess || !p)
                return STK_ERR_CUDA;
            g_scratch_addr[dev] = static_cast<double*>(p);
        }
        base = g_scratch_addr[dev];
    }
    // carve the workspace
    {
        long long off = 0;
        auto take = [&](long long cnt) {
            double* p = base + off;
            off = (off + cnt + 31) & ~31LL;
            return p;
        };
        for (int l = 0; l < nlev; ++l) {
            const Geom& g = L[l].g;
            L[l].C = stk::Coef<double>{};
            L[l].C.beta = take(g.nvel);
            L[l].C.invd_p = take(g.ncell);
            L[l].res = l + 1 < nlev ? take(g.ncell) : nullptr;   // coarsest: sweeps only
            L[l].phi = l > 0 ? take(g.ncell) : nullptr;
            L[l].rhs = l > 0 ? take(g.ncell) : nullptr;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int tpb = 256;
    k_na_fine_beta<<<(L[0].g.nvel + tpb - 1) / tpb, tpb, 0, s>>>(L[0].g, rho, L[0].C.beta);
    for (int l = 1; l < nlev; ++l)
        k_na_coarse_beta<<<(L[l].g.nvel + tpb - 1) / tpb, tpb, 0, s>>>(L[l - 1].g, L[l].g,
                                                                      L[l - 1].C.beta, L[l].C.beta);
    for (int l = 0; l < nlev; ++l)
        k_na_invdiag<<<(L[l].g.ncell + tpb - 1) / tpb, tpb, 0, s>>>(L[l].g, L[l].C.beta, L[l].C.invd_p);
    na_vcycle(L, nlev, 0, r_p, x_p, s);
    return cudaGetLastError() == cudaSuccess ? STK_OK : STK_ERR_CUDA;
}
