// Internal declarations shared by the translation units of libstokes_gb300.
//
// Geometry of one multigrid level of the staggered (MAC) grid, Sec. 3.1 of
// Cai et al., arXiv:1308.4605.  A velocity vector is stored "packed": the
// face arrays of components x, y[, z] one after the other (x fastest in each);
// a Stokes vector appends the cell array.  Wall faces are stored as zeros.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

namespace stk {

constexpr int PERIODIC = 0, NOSLIP = 1, FREESLIP = 2;

// Division by a run-time constant d >= 1 for 0 <= n < 2^31 (Granlund &
// Montgomery, round-up multiplier): n / d = (n * m) >> s.
struct FDiv {
    unsigned long long m;
    int s;
};
inline FDiv make_fdiv(int d) {
    FDiv f;
    if (d <= 1) {
        f.m = 1;
        f.s = 0;
        return f;
    }
    int l = 0;
    while ((1LL << l) < d) ++l;
    f.s = 32 + l;
    f.m = (unsigned long long)(((unsigned __int128)1 << f.s) / (unsigned)d) + 1;
    return f;
}
__host__ __device__ __forceinline__ int fdiv(int n, const FDiv& f) {
    return (int)(((unsigned long long)(unsigned)n * f.m) >> f.s);
}

struct Geom {
    int dim;
    int n[3];        // cells per axis (n[2] = 1 in 2D, or the instance count
                     // of a stacked 2D batch: instances along the third
                     // array axis, never coupled by a stencil)
    int nsl;         // instances stacked along the third axis (1 otherwise)
    int per[3];      // 1 if the axis is periodic
    int bclo[3];     // boundary code of the low side of each axis
    int bchi[3];
    int fe[3][3];    // extents (x, y, z) of the face array of component a
    int ee[3][3];    // extents of the edge array of pair p: 0=(x,y) 1=(x,z) 2=(y,z)
    int foff[3];     // offset of component a in a packed velocity vector
    int fsize[3];
    int esize[3];
    int nvel;        // length of a packed velocity vector
    int ncell;
    double h, ih, ih2;
    float ihf, ih2f;   // the same in FP32 (no FP64 conversion in FP32 kernels)
    // fast divisors: face extents fe[a][0], fe[a][1]; the colour row length
    // (fe[a][0]+1)/2; cell extents n[0], n[1]; the cell colour row n[0]/2
    FDiv fd_e0[3], fd_e1[3], fd_h0[3], fd_n0, fd_n1, fd_nh0;
};

// A packed Stokes vector of a stacked 2D batch: segment k (x faces, y faces,
// cells) holds the instances' values one after another, len[k] values each,
// starting at off[k]; nl = len[0] + len[1] + len[2] values per instance.
// Every length is even (power-of-two grids).
struct SliceMap {
    int len[3];
    int off[3];
    int nl;
};

// fill the derived fields of g (call after n, per, fe are set)
inline void finish_geom(Geom& g) {
    g.ihf = float(g.ih);
    g.ih2f = float(g.ih2);
    for (int a = 0; a < 3; ++a) {
        g.fd_e0[a] = make_fdiv(g.fe[a][0]);
        g.fd_e1[a] = make_fdiv(g.fe[a][1]);
        g.fd_h0[a] = make_fdiv((g.fe[a][0] + 1) / 2);
    }
    g.fd_n0 = make_fdiv(g.n[0]);
    g.fd_n1 = make_fdiv(g.n[1]);
    g.fd_nh0 = make_fdiv(g.n[0] / 2 > 0 ? g.n[0] / 2 : 1);
}

// Coefficients of one level (precision T).  alpha = theta rho_f and
// beta = 1/rho_f (coarsened by face averaging) are packed face vectors with
// zeros on wall faces; mu_e are the node (2D) / edge (3D) viscosities with
// zeros on free-slip walls and on edges lying on two walls; invd_u, invd_p
// are the inverse diagonals of A and L_rho.
template <typename T>
struct Coef {
    T* alpha;
    T* beta;
    T* mu2_c;    // 2 mu at cells: the factor of the normal stresses 2 mu du_a/dx_a
    T* mu_e[3];
    T* invd_u;
    T* invd_p;
    T* diag_u;   // the diagonal of A itself (FP64 hierarchy only; null in FP32)
    T* lam_c;    // bulk term gamma - 2/3 mu at cells; null without bulk viscosity
};

// Launch with programmatic dependent launch allowed: the kernel may be
// scheduled while its predecessor on the stream is still running; every
// kernel of this library starts with pdl_entry() (stencil.cuh), which lets
// its own dependents be scheduled and then waits until the predecessor grid
// has completed and its memory is visible.  Inside a captured graph the
// same holds through programmatic edges.  Semantics are those of ordinary
// stream order; only launch latency is hidden.
// launches issued by this host thread through launch_pdl: entry points that
// launch outside the profiled scopes (coefficient setup) add the difference
// to their handle's kernel count
inline thread_local long long tl_launches = 0;

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t s,
                              Args... args) {
    ++tl_launches;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// First statement of every kernel of this library: let the next kernel on
// the stream be scheduled, then wait until the previous grid has completed
// and its memory is visible (a no-op without programmatic dependent launch).
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Bounds-checked builds (nvcc -DSTK_BOUNDS_CHECK, `build.py --bounds-check`):
// the stencil index helpers check every index against the length of the
// array it addresses.  An index out of range is counted, the first one is
// recorded with its kind (1 face, 2 cell, 3 edge, 4 shared memory), and the
// access goes to element 0 instead, so it stays in bounds and the kernel
// runs to its end: no trap and no fault.  Each translation unit keeps its
// own record (module-local device variable) and exports a reader through
// STK_OOB_READER(name).  Release builds compile the checks away.
#ifdef STK_BOUNDS_CHECK
namespace {
__device__ unsigned long long g_oob[3];   // count, first kind, first index
}
__device__ __forceinline__ int chk_index(int i, int n, int kind) {
    if (i >= 0 && i < n) return i;
    if (atomicAdd(&g_oob[0], 1ull) == 0ull) {
        g_oob[1] = (unsigned long long)kind;
        g_oob[2] = (unsigned long long)(long long)i;
    }
    return 0;
}
#define STK_IDX(i, n, kind) ::stk::chk_index((i), (n), (kind))
// long long oob_<name>(long long first[2], int reset): this module's count
#define STK_OOB_READER(name)                                                          \
    long long oob_##name(long long first[2], int reset) {                             \
        unsigned long long v[3] = {0, 0, 0};                                          \
        if (cudaMemcpyFromSymbol(v, g_oob, sizeof v) != cudaSuccess) return -1;       \
        if (first && v[0]) {                                                          \
            first[0] = (long long)v[1];                                               \
            first[1] = (long long)v[2];                                               \
        }                                                                             \
        if (reset) {                                                                  \
            const unsigned long long z[3] = {0, 0, 0};                                \
            cudaMemcpyToSymbol(g_oob, z, sizeof z);                                   \
        }                                                                             \
        return (long long)v[0];                                                       \
    }
long long oob_kernels(long long first[2], int reset);
long long oob_pair(long long first[2], int reset);
long long oob_stress(long long first[2], int reset);
long long oob_coarse(long long first[2], int reset);
// a kernel that checks index n against length n (out of range by one)
// without any memory access: exercises the record in bounds-checked builds
void launch_oob_selftest(int n, cudaStream_t s);
#else
#define STK_IDX(i, n, kind) (i)
#define STK_OOB_READER(name)
#endif

// FP32 -> FP64, exact, with integer instructions (IEEE 754 binary32 ->
// binary64: same sign, exponent rebiased by 1023 - 127 = 896, fraction
// shifted left by 29).  The conversion instruction runs on GB300's FP64
// pipe, which streaming kernels that widen every element would otherwise
// saturate; zeros are built here too, and only subnormal, infinite and NaN
// inputs (exponent field 0 with a non-zero fraction, or 255) take the
// conversion instruction.
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    if (e == 0u || e == 0xffu) {
        if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)sign);
        return double(f);
    }
    const unsigned long long bits = sign | ((unsigned long long)(e + 896u) << 52) |
                                    ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double widen(double d) { return d; }

// zero n elements (a kernel, so that it takes part in the launch chain)
template <typename T>
void launch_zero(int n, T* x, cudaStream_t s);

// ---- launch wrappers (kernels.cu); all asynchronous on `s` -------------------

// coefficients
void launch_fine_coefficients(const Geom& g, const double* rho, const double* mu, double theta,
                              Coef<double> C, cudaStream_t s);
// lam = gamma - 2/3 mu on the cells of the finest level
void launch_bulk_lambda(int n, const double* gamma, const double* mu, double* lam, cudaStream_t s);
void launch_coarsen_coefficients(const Geom& gf, Coef<double> Cf, const Geom& gc, Coef<double> Cc,
                                 cudaStream_t s);
void launch_inverse_diagonals(const Geom& g, Coef<double> C, cudaStream_t s);
void launch_convert_coefficients(const Geom& g, Coef<double> C, Coef<float> Cf, cudaStream_t s);

// y = M x (packed Stokes vectors, FP64; y = b - M x when b is given) and the
// finest-level FP64 velocity residual, evaluated
// through stresses computed once per cell and edge (stress.cu); W holds the
// scratch stress arrays of the finest level (cells: dim arrays of ncell;
// edges: one array of esize[p] per pair p).
struct StressWork {
    double* tc[3];
    double* te[3];
};
void launch_stokes_matvec_stress(const Geom& g, Coef<double> C, const StressWork& W, const double* x,
                                 const double* b, double* y, cudaStream_t s);
void launch_vel_residual_stress(const Geom& g, Coef<double> C, const StressWork& W, const double* phi,
                                const double* rhs, double* res, bool after_sweep, cudaStream_t s);

// multigrid (precision T)
// first: this colour belongs to the first sweep from a zero initial guess
// (sweeps run red, then black, component by component), so the faces of the
// colour not yet swept and the later components are known to be zero
template <typename T>
void launch_vel_gs_colour(const Geom& g, Coef<T> C, int comp, int parity, T* phi, const T* rhs,
                          cudaStream_t s, int tpb = 256, bool first = false);   // tpb <= 512
template <typename T>
void launch_vel_residual(const Geom& g, Coef<T> C, const T* phi, const T* rhs, T* res,
                         cudaStream_t s, bool after_sweep = false);
template <typename T>
void launch_vel_restrict(const Geom& gf, const T* res, const Geom& gc, T* rhs_c, cudaStream_t s);
template <typename T>
void launch_vel_prolong_add(const Geom& gc, const T* phi_c, const Geom& gf, T* phi_f,
                            cudaStream_t s);
// both colours of one sweep, out of place (pair.cu): velocity component
// comp read from src (components < comp from dst) and written to dst
template <typename T>
void launch_vel_gs_pair(const Geom& g, Coef<T> C, int comp, const T* src, T* dst, const T* rhs,
                        cudaStream_t s);
template <typename T>
void launch_cell_gs_pair(const Geom& g, Coef<T> C, const T* src, T* dst, const T* rhs,
                         cudaStream_t s);
template <typename T>
void launch_cell_gs_colour(const Geom& g, Coef<T> C, int parity, T* phi, const T* rhs,
                           cudaStream_t s, int tpb = 256, bool first = false);  // tpb <= 512
template <typename T>
void launch_cell_residual(const Geom& g, Coef<T> C, const T* phi, const T* rhs, T* res,
                          cudaStream_t s, bool after_sweep = false);
template <typename T>
void launch_cell_restrict(const Geom& gf, const T* res, const Geom& gc, T* rhs_c, cudaStream_t s);
template <typename T>
void launch_cell_prolong_add(const Geom& gc, const T* phi_c, const Geom& gf, T* phi_f,
                             cudaStream_t s);

// All levels from the one given down to the coarsest, in one single-block
// launch (coarse.cu): L points to nlev device-resident level descriptors.
template <typename T>
struct CLevel {
    Geom g;
    Coef<T> C;
    T *phi_u, *rhs_u, *res_u, *phi_p, *rhs_p, *res_p;
    // coarsest level only: the matrices of its coarse solve (see
    // launch_coarsest_matrix) and the sweep count they hold (0: none)
    const T* smat_u = nullptr;
    const T* smat_p = nullptr;
    int smat_nc = 0;
};
// levels this small run in the coarse kernel: one SM's FP32 rate makes 4096
// cells (16^3, 64^2) worth it; its FP64 rate (1/152 of about 1.2 TFLOP/s)
// only 512 (8^3, 16x32)
constexpr int COARSE_MAX_CELLS_F32 = 4096;
constexpr int COARSE_MAX_CELLS_F64 = 512;
// nsl > 1: a stacked batch, one block per instance (these thresholds then
// apply to the cells of one instance)
template <typename T>
void launch_coarse_vcycle_vel(int dim, int nsl, const CLevel<T>* L, int nlev, const T* rhs, T* phi,
                              int nu, int ncoarse, bool bulk, size_t smem, cudaStream_t s);
template <typename T>
void launch_coarse_vcycle_cell(int dim, int nsl, const CLevel<T>* L, int nlev, const T* rhs, T* phi,
                               int nu, int ncoarse, size_t smem, cudaStream_t s);
// The same V-cycle from the level L[0] down as one persistent cooperative
// launch (coarse.cu): levels 0..lblock-1 as grid-wide stages separated by
// grid barriers (every block resident: one block of 1024 threads per SM at
// most, as many as the first level has points of one colour per 1024
// threads), levels lblock.. by one block.  Each barrier wait is bounded by
// *budget clock64() cycles (a device scalar, read at launch, so captured
// graphs follow changes); when one runs out, STK_ERR_TIMEOUT is written to
// *status and the launch ends at its next barriers.  bar: two unsigned words
// of device memory (zeroed before the launch, on s).  g0: L[0]'s geometry.
template <typename T>
cudaError_t launch_grid_vcycle_vel(int dim, const Geom& g0, const CLevel<T>* L, int nlev, int lblock,
                                   const T* rhs, T* phi, int nu, int ncoarse, bool bulk, unsigned* bar,
                                   const long long* budget, int* status, cudaStream_t s);
template <typename T>
cudaError_t launch_grid_vcycle_cell(int dim, const Geom& g0, const CLevel<T>* L, int nlev, int lblock,
                                    const T* rhs, T* phi, int nu, int ncoarse, unsigned* bar,
                                    const long long* budget, int* status, cudaStream_t s);
// Stacked batches, shared-memory variant: block s runs instance s through
// the descriptors Lall[s * lstride + l] (one instance's geometry and
// coefficients); rhs, phi in the stacked layout (coarse.cu)
template <typename T>
void launch_coarse_stacked(bool vel, int dim, int nsl, const CLevel<T>* Lall, int lstride, int nlev,
                           const T* rhs, T* phi, int nu, int ncoarse, bool bulk, size_t smem,
                           cudaStream_t s);
// dst[s * gl.nvel + i] = the i-th face value of instance s of the stacked
// face array src (gl: the geometry of one instance)
template <typename T>
void launch_faces_by_instance(const Geom& gl, int nsl, const T* src, T* dst, cudaStream_t s);
// The same as one thread-block cluster (up to 16 CTAs of 1024 threads on one
// GPC, as many as the level's size calls for): hardware cluster barriers
// between the stages (coarse.cu).  Not for stacked batches.
template <typename T>
cudaError_t launch_cluster_vcycle_vel(int dim, const Geom& g0, const CLevel<T>* L, int nlev, int lblock,
                                      const T* rhs, T* phi, int nu, int ncoarse, bool bulk, cudaStream_t s);
template <typename T>
cudaError_t launch_cluster_vcycle_cell(int dim, const Geom& g0, const CLevel<T>* L, int nlev, int lblock,
                                       const T* rhs, T* phi, int nu, int ncoarse, cudaStream_t s);
// Shared-memory budget of the coarse-level kernels: with smem > 0 (the bytes
// of phi, rhs and residual of every level handled) and at most this many
// bytes, the work vectors live in shared memory; 0 keeps them in global
// memory.  prepare_coarse_kernels() raises the kernels' dynamic shared-memory
// limit on the current device.
constexpr size_t COARSE_SMEM_LIMIT = 220 * 1024;
void prepare_coarse_kernels();

// The coarse solve of App. C, ncoarse Gauss-Seidel sweeps on the coarsest
// level from a zero initial guess, is a fixed linear map phi = S rhs of that
// level's n unknowns (n = faces, or cells).  For n <= SMAT_MAX it is formed
// once per coefficient set, column i from the same sweeps applied to the
// unit vector e_i (stored column-major: st[i * n + j] = S_ji), and then
// applied as a matrix: one short parallel stage instead of 6 ncoarse
// (velocity) or 2 ncoarse (pressure) dependent ones.  The two agree up to
// rounding.
constexpr int SMAT_MAX = 1024;
template <typename T>
void launch_coarsest_matrix_vel(const Geom& g, Coef<T> C, int ncoarse, T* st, cudaStream_t s);
template <typename T>
void launch_coarsest_matrix_cell(const Geom& g, Coef<T> C, int ncoarse, T* st, cudaStream_t s);
// phi = S rhs (one block; the same sums, in the same order, as inside the
// coarse-level kernel)
template <typename T>
void launch_coarsest_apply(int n, const T* st, const T* rhs, T* phi, cudaStream_t s);

// preconditioner algebra (precision T)
template <typename T>  // bc = D u + bp
void launch_div_plus(const Geom& g, const T* u, const T* bp, T* bc, cudaStream_t s);
template <typename T>  // out = u - beta G p (beta may be null: out = u - G p)
void launch_sub_grad(const Geom& g, const T* beta, const T* u, const T* p, T* out, cudaStream_t s);
template <typename T>  // out = b - G p - A u
void launch_vel_correction_rhs(const Geom& g, Coef<T> C, const T* b, const T* p, const T* u,
                               T* out, cudaStream_t s);
template <typename T>  // xp = theta phi - (mu2 + lam) bc, mu2 = 2 mu  (phi, lam may be null)
void launch_schur_combine(int n, const double* theta, const T* phi, const T* mu2, const T* lam,
                          const T* bc, T* xp,
                          cudaStream_t s);

// Device-resident state of restarted GMRES (gmres.cu): the rotated
// Hessenberg matrix, the Givens rotations, the rotated right-hand side g, the
// least-squares solution y, the residuals and the stopping decisions of the
// current cycle.  cond[] holds the decisions that gate the next phase: the
// stopping test of a cycle (GM_COND_CHK, open while the solve runs), its
// preconditioned start (GM_COND_PRE), its final update (GM_COND_FIN) and
// Arnoldi step j (GM_COND_STEP0 + j).
constexpr int GM_MMAX = 32;
constexpr int GM_NHIST = 256;    // true relative residuals at cycle starts kept
constexpr int GM_NEST = 2048;    // Arnoldi residual estimates kept
constexpr int GM_COND_PRE = 0, GM_COND_FIN = 1, GM_COND_CHK = 2, GM_COND_STEP0 = 3;
constexpr int GM_NCOND = GM_COND_STEP0 + GM_MMAX;
enum { GM_RUNNING = 0, GM_CONVERGED = 1, GM_MAXIT = 2, GM_NONFINITE = 3, GM_TIMEOUT = 4 };
enum { GM_WHY_RHS = 1, GM_WHY_RESIDUAL, GM_WHY_PRECOND, GM_WHY_ARNOLDI, GM_WHY_UPDATE };
struct GmState {
    // header: read by the host after every cycle
    int state, why, k, iterations, restarts, maxit, m, flex, nhist, nest;
    int wait_status;   // STK_ERR_TIMEOUT once a bounded device wait ran out, else 0
    double bnorm, rnorm, beta, target, est, rtol, inv_scale;
    unsigned cond[GM_NCOND];
    // column j of H at H[j * (GM_MMAX + 1)], rows 0..j+1
    double H[(GM_MMAX + 1) * GM_MMAX];
    double cs[GM_MMAX], sn[GM_MMAX], g[GM_MMAX + 1], y[GM_MMAX];
    double hist[GM_NHIST];       // ||b - M x|| / ||b|| at each cycle start
    double est_hist[GM_NEST];    // |g_{j+1}| / ||b|| after each Arnoldi step
};
// solve start (*bn2 = ||b||^2), cycle start (*rn2 = ||b - M x||^2), first
// basis vector (*vn2 = ||P^{-1} r||^2 for the left form), Arnoldi step j
// (hcol[0..j] the projections, *n2 = ||w||^2 after them), cycle end.  st
// holds nsl records (a stacked batch: one per instance), instance y's
// scalars at y * dstride; gc[GM_NCOND] receives the OR of the instances'
// decisions.  With use != 0 that OR is also written to the graph's
// conditional handle.
void launch_gm_begin(GmState* st, int nsl, unsigned* gc, const double* bn2, int dstride, double rtol,
                     int maxit, int m, int flex, cudaStream_t s);
void launch_gm_check(GmState* st, int nsl, unsigned* gc, const double* rn2, int dstride,
                     cudaGraphConditionalHandle hpre, int use, cudaStream_t s);
// graph only: open the cycle's stopping test while an instance is running
void launch_gm_gate(GmState* st, int nsl, unsigned* gc, cudaGraphConditionalHandle hchk, cudaStream_t s);
void launch_gm_start(GmState* st, int nsl, unsigned* gc, const double* vn2, int dstride,
                     cudaGraphConditionalHandle h0, int use0, cudaGraphConditionalHandle hfin, int usefin,
                     cudaStream_t s);
void launch_gm_step(GmState* st, int nsl, unsigned* gc, int j, const double* hcol, const double* n2,
                    int dstride, cudaGraphConditionalHandle hn, int use, cudaStream_t s);
void launch_gm_finish(GmState* st, int nsl, cudaStream_t s);

// reductions with a fixed block count: deterministic results
constexpr int RED_BLOCKS = 304;   // 2 x 152 SMs
constexpr int RED_THREADS = 256;
constexpr int KRY_BLOCKS = 1216;  // 8 x 152 SMs: grid of the Krylov kernels (krylov.cu)
constexpr int RED_SCRATCH = KRY_BLOCKS * 36;   // doubles of reduction scratch
// Reductions finish in the last block of their own launch: cnt is a count
// in device memory, zero between reductions, one per stream that reduces
// (per instance for the stacked forms).
template <typename T>  // out[0] = sum x, out[1] = out[0] / n  (scratch >= RED_BLOCKS doubles)
void launch_sum(int n, const T* x, double* scratch, double* out, unsigned* cnt, cudaStream_t s);
// the same for an FP32 vector, x 16-byte aligned (krylov.cu; scratch >=
// KRY_BLOCKS doubles): wide loads, sums of four in FP32 widened once
void launch_sum_f32x4(int n, const float* x, double* scratch, double* out, unsigned* cnt, cudaStream_t s);
template <typename T>  // x -= sum[1] (the mean left by launch_sum)
void launch_sub_mean(int n, T* x, const double* sum, cudaStream_t s);
template <typename T>  // out = in - sum[1]
void launch_copy_sub_mean(int n, const T* in, T* out, const double* sum, cudaStream_t s);
// Stacked batches: nsl instances of n values one after another.
// out[y * ostride] = sum of instance y, out[y * ostride + 1] its mean,
// bitwise the values launch_sum gives for that instance alone (scratch >=
// nsl * RED_BLOCKS doubles; cnt: nsl counts)
template <typename T>
void launch_sum_sl(int n, int nsl, const T* x, double* scratch, double* out, int ostride, unsigned* cnt,
                   cudaStream_t s);
// out = in - sum[y * stride + 1] per instance y (in == out allowed)
template <typename T>
void launch_sub_mean_sl(int n, int nsl, const T* in, T* out, const double* sum, int stride, cudaStream_t s);
// j = 0: h[0] = <w, V[0]>; j = -1: h[0] = <w, w> (V unused)
void launch_multidot(int n, int j, const double* const* V, const double* w, double* scratch,
                     double* h, unsigned* cnt, cudaStream_t s);
// modified Gram-Schmidt step: w -= h[k] vk, then out[0] = <w, u> (u = null: <w, w>)
void launch_mgs_step(int n, const double* vk, const double* u, const double* h, int k, double* w,
                     double* scratch, double* out, unsigned* cnt, cudaStream_t s);
// x += sum_i y[i] V_i (i < k); V of precision TV
template <typename TV>
void launch_combine(int n, int k, const TV* const* V, const double* y, double* x, cudaStream_t s);
// x += sum_i y[i] V_i for i < *k (k read on the device, 0 <= *k <= m <= 32;
// the vectors beyond *k are not read)
template <typename TV>
void launch_combine_dev(int n, int m, const TV* const* V, const double* y, const int* k, double* x,
                        cudaStream_t s);
// x *= *a (a device scalar)
void launch_scale_dev(int n, double* x, const double* a, cudaStream_t s);
// Stacked batches (krylov.cu): the calls above on every instance of the
// batch (nsl instances, map m), instance y's results at stride hstride /
// ostride (y * stride + k), bitwise the ones it gets alone.
void launch_multidot_sl(const SliceMap& m, int nsl, int j, const double* const* V, const double* w,
                        double* scratch, double* h, int hstride, unsigned* cnt, cudaStream_t s);
void launch_mgs_step_sl(const SliceMap& m, int nsl, const double* vk, const double* u, const double* h,
                        int hstride, int k, double* w, double* scratch, double* out, int ostride,
                        unsigned* cnt, cudaStream_t s);
// x += sum_i st[y].y[i] V_i (i < st[y].k) for every instance y
template <typename TV>
void launch_combine_dev_sl(const SliceMap& m, int nsl, int mmax, const TV* const* V, const GmState* st,
                           double* x, cudaStream_t s);
// x *= st[y].inv_scale where Arnoldi step j of instance y is open, else 0
void launch_scale_dev_sl(const SliceMap& m, int nsl, double* x, const GmState* st, int j, cudaStream_t s);
// out[y * ostride] = sum of instance y of an FP32 vector of nsl x n values,
// out[y * ostride + 1] its mean
void launch_sum_f32x4_sl(int n, int nsl, const float* x, double* scratch, double* out, int ostride,
                         unsigned* cnt, cudaStream_t s);
// x *= 1 / sqrt(*nrm2)
void launch_scale_inv_sqrt(int n, double* x, const double* nrm2, cudaStream_t s);
void launch_scale(int n, double* x, double a, cudaStream_t s);
template <typename T>  // y += a x
void launch_axpy(int n, T a, const T* x, T* y, cudaStream_t s);
template <typename TA, typename TB>
void launch_convert(int n, const TA* a, TB* b, cudaStream_t s);
// dL/dlog mu and dL/drho (cell arrays) from packed velocities u and lambda
// inhomogeneous boundary data: wall faces of src into the packed dst; the
// tangential-velocity terms of a no-slip wall subtracted from c
void launch_copy_walls(const Geom& g, int a, const double* src, double* dst, cudaStream_t s);
void launch_wall_tangential(const Geom& g, const double* mu_e, int d, int side, int a,
                            const double* U, double* c, cudaStream_t s);
// b = alpha u + f on the a-faces (f may be null), zero on wall faces
void launch_inertial_rhs(const Geom& g, int a, const double* alpha, const double* u,
                         const double* f, double* b, cudaStream_t s);
void launch_gradient(const Geom& g, const double* mu, double theta, const double* u,
                     const double* lam, double* glogmu, double* grho, cudaStream_t s);
// out[0] = number of non-finite entries, out[1] = number of entries <= 0
void launch_check_fields(int n, const double* rho, const double* mu, double* scratch, double* out,
                         cudaStream_t s);

}  // namespace stk
