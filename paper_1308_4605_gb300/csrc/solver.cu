// Host side of libstokes_gb300: the multigrid hierarchy, the V-cycles
// (App. C), the block preconditioners P1..P5 (Sec. 2), restarted GMRES
// (Sec. 3.2) and flexible GMRES with an FP32 preconditioner (Sec. 4), and the
// C ABI declared in include/stokes.h.
//
// Reference: Cai, Nonaka, Bell, Griffith & Donev, arXiv:1308.4605.
#include "internal.cuh"
#include "../../include/stokes.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

using namespace stk;

namespace {

thread_local std::string g_create_error;

// NVTX range over a host-side phase (visible to Nsight tools; a no-op
// without an attached tool)
struct Nvtx {
    explicit Nvtx(const char* name) { nvtxRangePushA(name); }
    ~Nvtx() { nvtxRangePop(); }
    Nvtx(const Nvtx&) = delete;
    Nvtx& operator=(const Nvtx&) = delete;
};

struct ProfRec {
    int cat;
    double bytes;
    double flops;
    cudaEvent_t a, b;
};

const char* kProfNames[STK_NPROF] = {
    "stokes_matvec",    "vel_smooth_colour", "vel_residual",  "vel_restrict",
    "vel_prolong_add",  "cell_smooth_colour", "cell_residual", "cell_restrict",
    "cell_prolong_add", "precond_algebra",   "mean_removal",  "arnoldi_multidot",
    "arnoldi_update",   "krylov_combine",    "convert",       "coarse_levels",
    "vel_smooth_colour_l0", "cell_smooth_colour_l0", "vel_smooth_pair_l0", "vel_smooth_pair",
    "cell_smooth_pair_l0", "cell_smooth_pair", "vel_smooth_first", "cell_smooth_first"};

enum {
    PF_MATVEC = 0, PF_VSMOOTH, PF_VRES, PF_VRESTR, PF_VPROL, PF_CSMOOTH, PF_CRES, PF_CRESTR,
    PF_CPROL, PF_ALG, PF_MEAN, PF_MDOT, PF_UPD, PF_COMB, PF_CONV, PF_COARSE, PF_VSMOOTH0,
    PF_CSMOOTH0, PF_VPAIR0, PF_VPAIR, PF_CPAIR0, PF_CPAIR, PF_VFIRST, PF_CFIRST
};

template <typename T>
struct Work {            // multigrid work vectors of one level
    T *phi_u, *rhs_u, *res_u, *phi_p, *rhs_p, *res_p;
    T *alt_u, *alt_p;    // second buffers of the out-of-place two-colour sweeps
};

struct Level {
    Geom g;
    Coef<double> cd;
    Coef<float> cf;
    Work<double> wd;
    Work<float> wf;
    double* lam_d = nullptr;   // storage of the bulk term (allocated on first use)
    float* lam_f = nullptr;
    // coarsest level only: the coarse-solve matrices (launch_coarsest_matrix),
    // allocated when the level has at most SMAT_MAX faces (cells)
    double* smat_ud = nullptr;
    double* smat_pd = nullptr;
    float* smat_uf = nullptr;
    float* smat_pf = nullptr;
    // stacked batches, levels from lstk on: the geometry of one instance, its
    // face coefficients copied instance by instance (cell and edge arrays
    // already hold the instances one after another) and, on the coarsest
    // level, one coarse-solve matrix per instance
    Geom gi{};
    Coef<double> cdi{};
    Coef<float> cfi{};
    double *smat_udi = nullptr, *smat_pdi = nullptr;
    float *smat_ufi = nullptr, *smat_pfi = nullptr;
};

// the sweep count the coarse-solve matrices are formed for: the default
// ncoarse (App. C); other counts sweep
constexpr int SMAT_SWEEPS = 8;
template <typename T> const T* smat_u_of(const Level& L);
template <> const double* smat_u_of<double>(const Level& L) { return L.smat_ud; }
template <> const float* smat_u_of<float>(const Level& L) { return L.smat_uf; }
template <typename T> const T* smat_p_of(const Level& L);
template <> const double* smat_p_of<double>(const Level& L) { return L.smat_pd; }
template <> const float* smat_p_of<float>(const Level& L) { return L.smat_pf; }

template <typename T>
struct PBuf {            // level-0 buffers of the preconditioner in precision T
    T* in;               // packed Stokes input (mixed form: converted Krylov vector)
    T* bc;               // cell: D x* + b_p
    T* tmpu;             // velocity temporary
    T* xs;               // velocity x*
    T *ru, *du;          // velocity residual and correction of repeated V-cycles
    T *rp, *dp;          // the same for the pressure
};

}  // namespace

struct stk_handle {
    int device = 0;
    int dim = 0;
    // a stacked batch (2D): nsl instances of one grid along the third array
    // axis of every array; smap locates an instance in a packed vector
    int nsl = 1;
    SliceMap smap{};
    std::vector<Level> lev;
    double theta = 0.0;
    bool coef_set = false;
    std::string err;
    std::vector<void*> allocs;
    PBuf<double> pd{};
    PBuf<float> pf{};
    int m_alloc = 0;
    std::vector<double*> V;
    std::vector<float*> Z;
    double *bk = nullptr, *xk = nullptr, *tmp = nullptr;
    int lcoarse_d = 0, lcoarse_f = 0;        // first level run by the coarse kernel (FP64, FP32)
    int tpb_d = 256, tpb_f = 256;            // threads per block of the colour kernels
    int lpair_d = 0, lpair_f = 0;            // first level smoothed by the two-colour kernels
    int lgrid_d = 0, lgrid_f = 0;            // first level run by the persistent multi-block kernel
    int lcluster_d = 0, lcluster_f = 0;      // first level run by the thread-block-cluster kernel
    unsigned* gbar = nullptr;                // its grid barrier (two words), then the wait
                                             // budget in clock64() cycles (a long long)
    bool bulk = false;                       // bulk-viscosity stress form on
    StressWork sw{};                         // stress scratch of the finest level (FP64)
    double *gamma = nullptr, *rho0 = nullptr, *mu0 = nullptr;   // level-0 fields
    CLevel<double>* cld = nullptr;           // device copies of the level descriptors
    CLevel<float>* clf = nullptr;
    // stacked batches: descriptors of one instance's levels lstk.. for the
    // shared-memory coarse-level kernel, instance s at s * (levels - lstk)
    int lstk = 0;
    CLevel<double>* clsd = nullptr;
    CLevel<float>* clsf = nullptr;
    double* red = nullptr;    // reduction scratch (RED_BLOCKS * 36 doubles)
    unsigned* rcnt = nullptr; // counts of the reductions' last blocks (one per instance)
    double* dsc = nullptr;    // device scalars
    double* hpin = nullptr;   // pinned host staging
    bool prof = false;
    long long nkern = 0;      // kernels launched by this handle
    // CUDA graphs of preconditioner applications, keyed by
    // (which, sizeof(T), input, output, nu, ncoarse, profiling)
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        long long kernels = 0;
        std::vector<ProfRec> recs;   // event pairs captured inside (profiling)
    };
    std::map<std::tuple<int, int, const void*, void*, int, int, int, int>, GraphEntry> graphs;
    bool use_graphs = true;
    bool capturing = false;
    long long cap_kernels = 0;
    std::vector<ProfRec> caprecs;
    cudaStream_t cap = nullptr;    // private stream used for capture only
    cudaStream_t run = nullptr;    // this handle's stream inside a batched solve
    cudaEvent_t join = nullptr;    // marks the end of its work in a batched solve
    cudaEvent_t cyc = nullptr;     // marks the end of a GMRES cycle (header read included)
    // graphs of one GMRES cycle (conditional nodes gate its phases), keyed by
    // (precond, flexible, m, nu, ncoarse, cycles); kernels per phase
    struct CycleGraph {
        cudaGraphExec_t exec = nullptr;
        long long k_gate = 0, k_chk = 0, k_pre = 0, k_fin = 0;
        std::vector<long long> k_step;
    };
    std::map<std::tuple<int, int, int, int, int, int>, CycleGraph> cgraphs;
    // graphs of single phases of a cycle (host-gated batches), keyed by
    // (phase, precond, flexible, m, nu, ncoarse, cycles); kernels each
    std::map<std::tuple<int, int, int, int, int, int, int>, std::pair<cudaGraphExec_t, long long>> pgraphs;

    GmState* gst = nullptr;        // device state of the GMRES least-squares problem (one per instance)
    GmState* gst_host = nullptr;   // pinned copy
    unsigned* gcond = nullptr;     // the OR of the instances' decisions (device)
    unsigned* gcond_host = nullptr;
    std::vector<stk_solve_info> sinfo;          // per instance, last solve
    std::vector<int> sit_before;                // iterations before the current cycle
    std::vector<std::vector<double>> hist_true, hist_est;   // residual histories of the last solve
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> evpool;
    size_t evnext = 0;
    long long plaunch[STK_NPROF] = {};
    double pms[STK_NPROF] = {}, pbytes[STK_NPROF] = {}, pflops[STK_NPROF] = {};
};

namespace {

constexpr int NDSC = 128;     // device scalar slots
// batches of at most this many handles run one cycle graph per handle
constexpr int BATCH_CYCLE_GRAPHS = 8;
// slots of h->dsc
constexpr int DS_SUM = 0;     // mean removal sums
constexpr int DS_H = 8;       // Arnoldi column h[0..m+1]
constexpr int DS_N2 = 48;     // norms
constexpr int DS_THETA = 100; // theta = 1/dt (read by the preconditioner graphs)
constexpr int HP_THETA = 250; // pinned host staging slot of theta

int fail(stk_handle* h, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_create_error = buf;
    return code;
}

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(h, STK_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

#define CKL()                                                                          \
    do {                                                                               \
        cudaError_t e_ = cudaGetLastError();                                           \
        if (e_ != cudaSuccess)                                                         \
            return fail(h, STK_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
cudaError_t dalloc(stk_handle* h, T** p, size_t n) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * (n ? n : 1));
    if (e != cudaSuccess) return e;
    h->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return cudaMemset(q, 0, sizeof(T) * (n ? n : 1));
}

// nsl > 1 (2D only): nsl instances of the grid stacked along the third
// array axis (a stacked batch)
Geom make_geom(int dim, const int n[3], double hh, const int bc[6], int nsl = 1) {
    Geom g{};
    g.dim = dim;
    g.nsl = dim == 2 ? nsl : 1;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = a < dim ? n[a] : (a == 2 ? g.nsl : 1);
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
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    for (int p = 0; p < 3; ++p) {
        for (int c = 0; c < 3; ++c)
            g.ee[p][c] = g.n[c] + (((c == pa[p] || c == pb[p]) && !g.per[c]) ? 1 : 0);
        g.esize[p] = pb[p] < dim ? g.ee[p][0] * g.ee[p][1] * g.ee[p][2] : 0;
    }
    g.h = hh;
    g.ih = 1.0 / hh;
    g.ih2 = 1.0 / (hh * hh);
    stk::finish_geom(g);
    return g;
}

// -------------------------------------------------------------------- profiling
struct Scope {
    stk_handle* h;
    ProfRec rec{};
    cudaStream_t s;
    Scope(stk_handle* h_, int cat, double bytes, cudaStream_t s_, int kernels = 1,
          double flops = 0.0)
        : h(h_), s(s_) {
        if (h->capturing) h->cap_kernels += kernels;
        else h->nkern += kernels;
        if (!h->prof) return;
        rec.cat = cat;
        rec.bytes = bytes;
        rec.flops = flops;
        rec.a = next_event();
        rec.b = next_event();
        record(rec.a);
    }
    ~Scope() {
        if (!h->prof) return;
        record(rec.b);
        if (h->capturing) h->caprecs.push_back(rec);
        else h->recs.push_back(rec);
    }
    void record(cudaEvent_t e) {
        // inside a capture, an external record makes a timing event node
        if (h->capturing) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
        else cudaEventRecord(e, s);
    }
    cudaEvent_t next_event() {
        if (h->capturing) {   // events recorded by graph nodes belong to the graph
            cudaEvent_t e;
            cudaEventCreate(&e);
            return e;
        }
        if (h->evnext >= h->evpool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            h->evpool.push_back(e);
        }
        return h->evpool[h->evnext++];
    }
};

void prof_flush(stk_handle* h) {
    if (h->recs.empty()) return;
    cudaDeviceSynchronize();
    for (auto& r : h->recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        h->plaunch[r.cat] += 1;
        h->pms[r.cat] += ms;
        h->pbytes[r.cat] += r.bytes;
        h->pflops[r.cat] += r.flops;
    }
    h->recs.clear();
    h->evnext = 0;
}

// Algorithmic bytes of one launch: every input word read once, every output
// word written once.
double esum(const Geom& g) { return double(g.esize[0]) + g.esize[1] + g.esize[2]; }
template <typename T>
double bytes_vel_colour(const Geom& g, int a) {
    double e = 0;
    for (int b = 0; b < g.dim; ++b)
        if (b != a) e += g.esize[a + b - 1];
    // half of comp a: rhs and invd read and phi written; phi of all
    // components, mu2_c and the edge viscosities of comp a read
    return sizeof(T) * (1.5 * g.fsize[a] + g.nvel + g.ncell + e);
}
template <typename T>
double bytes_vel_residual(const Geom& g) {   // phi, rhs, alpha read; res written
    return sizeof(T) * (4.0 * g.nvel + g.ncell + esum(g));
}
template <typename T>
double bytes_cell_colour(const Geom& g) {    // half: rhs, invd, write; phi, beta all
    return sizeof(T) * (1.5 * g.ncell + g.ncell + g.nvel);
}
// The colours of the first sweep from zero read only what is not known to be
// zero (k_vel_gs with its zero mask): the half of comp a (rhs and the
// inverse diagonal read, phi written) always; phi_a unless its other colour
// is still zero; phi_b of the components already swept; mu2_c and the edge
// viscosities wherever a term needs them.
template <typename T>
double bytes_vel_first(const Geom& g, int a, int parity) {
    const bool za = parity == 0;
    double w = 1.5 * g.fsize[a] + (za ? 0.0 : g.fsize[a] + g.ncell);
    for (int b = 0; b < g.dim; ++b) {
        if (b == a) continue;
        const bool zb = b > a;
        if (!zb) w += g.fsize[b];
        if (!(za && zb)) w += g.esize[a + b - 1];
    }
    return sizeof(T) * w;
}
template <typename T>
double bytes_cell_first(const Geom& g) {   // red from zero: rhs, invd half, write half
    return sizeof(T) * 1.5 * g.ncell;
}
// kernels of one stress-based operator or residual evaluation: cells, one
// per edge family, faces
int stress_kernels(const Geom& g) { return g.dim == 3 ? 5 : 3; }

double bytes_matvec(const Geom& g, int in_size) {
    return in_size * double(g.nvel + g.ncell) + 8.0 * (2.0 * g.nvel + 2.0 * g.ncell + esum(g));
}

// --------------------------------------------------------------------- V-cycles
template <typename T> Coef<T> coef_of(const Level& L);
template <> Coef<double> coef_of<double>(const Level& L) { return L.cd; }
template <> Coef<float> coef_of<float>(const Level& L) { return L.cf; }
template <typename T> Work<T> work_of(const Level& L);
template <> Work<double> work_of<double>(const Level& L) { return L.wd; }
template <> Work<float> work_of<float>(const Level& L) { return L.wf; }
template <typename T> int lcoarse_of(const stk_handle* h) {
    return sizeof(T) == 8 ? h->lcoarse_d : h->lcoarse_f;
}
template <typename T> int tpb_of(const stk_handle* h) { return sizeof(T) == 8 ? h->tpb_d : h->tpb_f; }
template <typename T> int lgrid_of(const stk_handle* h) { return sizeof(T) == 8 ? h->lgrid_d : h->lgrid_f; }
template <typename T> int lcluster_of(const stk_handle* h) {
    return sizeof(T) == 8 ? h->lcluster_d : h->lcluster_f;
}
template <typename T> int lpair_of(const stk_handle* h) {
    return sizeof(T) == 8 ? h->lpair_d : h->lpair_f;
}
template <typename T> const CLevel<T>* clstk_of(const stk_handle* h);
template <> const CLevel<double>* clstk_of<double>(const stk_handle* h) { return h->clsd; }
template <> const CLevel<float>* clstk_of<float>(const stk_handle* h) { return h->clsf; }
template <typename T> const CLevel<T>* clev_of(const stk_handle* h);
template <> const CLevel<double>* clev_of<double>(const stk_handle* h) { return h->cld; }
template <> const CLevel<float>* clev_of<float>(const stk_handle* h) { return h->clf; }
template <typename T> PBuf<T>& pbuf_of(stk_handle* h);
template <> PBuf<double>& pbuf_of<double>(stk_handle* h) { return h->pd; }
template <> PBuf<float>& pbuf_of<float>(stk_handle* h) { return h->pf; }

// Bytes of phi, rhs and residual of levels l.. (faces or cells) if they fit
// the coarse kernel's shared-memory budget, else 0 (global-memory variant).
template <typename T>
size_t coarse_smem(const stk_handle* h, int l, bool vel) {
    const int nl = (int)h->lev.size();
    if (nl - l > 16) return 0;
    size_t b = 0;
    for (int k = l; k < nl; ++k)
        b += 3 * sizeof(T) * (size_t)(vel ? h->lev[k].g.nvel : h->lev[k].g.ncell);
    return b <= COARSE_SMEM_LIMIT ? b : 0;
}

// The same for one instance of a stacked batch (the shared-memory kernel
// runs each instance in its own block); 0 when the levels have no
// instance copies or do not fit.
template <typename T>
size_t coarse_smem_stk(const stk_handle* h, int l, bool vel) {
    const int nl = (int)h->lev.size();
    if (h->nsl == 1 || l < h->lstk || nl - l > 16) return 0;
    size_t b = 0;
    for (int k = l; k < nl; ++k)
        b += 3 * sizeof(T) * (size_t)(vel ? h->lev[k].gi.nvel : h->lev[k].gi.ncell);
    return b <= COARSE_SMEM_LIMIT ? b : 0;
}

struct MGParams {
    int nu = 2;
    int ncoarse = 8;
    int cu = 1;   // V-cycles per velocity subsolve
    int cp = 1;   // V-cycles per pressure subsolve
};

// Floating-point operations of one Gauss-Seidel point update (adds + muls +
// 2 x fmas), counted with ncu (sm__sass_thread_inst_executed_op_*) on the
// 3D kernels: velocity FP64 22 (16 instructions), FP32 24, cell 15 in both
// precisions (both multiply by the stored inverse diagonal); the 2D velocity
// stencil has one transverse axis instead of two (8 fewer operations).
template <typename T>
double flops_vel_point(int dim) {
    const double f3 = sizeof(T) == 8 ? 22.0 : 24.0;
    return dim == 3 ? f3 : f3 - 8.0;
}
double updated_faces(const Geom& g, int a) {   // unknown a-faces of one colour
    double n = double(g.fe[a][0]) * g.fe[a][1] * g.fe[a][2];
    if (!g.per[a]) n -= 2.0 * double(g.fsize[a]) / g.fe[a][a];
    return 0.5 * n;
}

template <typename T>
double bytes_vel_pair(const Geom& g, int a) {
    double e = 0;
    for (int b = 0; b < g.dim; ++b)
        if (b != a) e += g.esize[a + b - 1];
    // comp a: rhs and the inverse diagonal read and phi written; phi of
    // all components, mu2_c and the edge viscosities of comp a read
    return sizeof(T) * (3.0 * g.fsize[a] + g.nvel + g.ncell + e);
}

// nsweep Gauss-Seidel sweeps of the velocity on level l.  From the level
// lpair on, pairs of sweeps run as out-of-place two-colour kernels that
// alternate between phi and the level's second buffer (an even count ends
// in phi); an odd last sweep, and levels below lpair, use one launch per
// colour in place.
template <typename T>
void vel_sweeps(stk_handle* h, int l, int nsweep, T* phi, const T* rhs, cudaStream_t s,
                bool from_zero = false) {
    const Level& L = h->lev[l];
    Coef<T> C = coef_of<T>(L);
    const bool fine = l == 0;
    const double fl = flops_vel_point<T>(L.g.dim);
    int it = 0;
    if (l >= lpair_of<T>(h)) {
        T* buf[2] = {phi, work_of<T>(L).alt_u};
        for (; it < (nsweep & ~1); ++it)
            for (int a = 0; a < L.g.dim; ++a) {
                Scope sc(h, fine ? PF_VPAIR0 : PF_VPAIR, bytes_vel_pair<T>(L.g, a), s, 1,
                         2.0 * fl * updated_faces(L.g, a));
                launch_vel_gs_pair<T>(L.g, C, a, buf[it & 1], buf[(it + 1) & 1], rhs, s);
            }
    }
    for (; it < nsweep; ++it)
        for (int a = 0; a < L.g.dim; ++a)
            for (int par = 0; par < 2; ++par) {
                // the first sweep from zero skips the terms of zero values
                // (plain form only; with bulk viscosity every sweep is full)
                const bool first = from_zero && it == 0 && !h->bulk;
                if (first) {
                    Scope sc(h, PF_VFIRST, bytes_vel_first<T>(L.g, a, par), s, 1, 0.0);
                    launch_vel_gs_colour<T>(L.g, C, a, par, phi, rhs, s, tpb_of<T>(h), true);
                    continue;
                }
                Scope sc(h, fine ? PF_VSMOOTH0 : PF_VSMOOTH, bytes_vel_colour<T>(L.g, a), s, 1,
                         fl * updated_faces(L.g, a));
                launch_vel_gs_colour<T>(L.g, C, a, par, phi, rhs, s, tpb_of<T>(h));
            }
}

template <typename T>
void cell_sweeps(stk_handle* h, int l, int nsweep, T* phi, const T* rhs, cudaStream_t s,
                 bool from_zero = false) {
    const Level& L = h->lev[l];
    Coef<T> C = coef_of<T>(L);
    const bool fine = l == 0;
    const double fl = 15.0 * 0.5 * L.g.ncell;
    int it = 0;
    if (l >= lpair_of<T>(h)) {
        T* buf[2] = {phi, work_of<T>(L).alt_p};
        for (; it < (nsweep & ~1); ++it) {
            // rhs and inverse diagonal read, phi read and written, beta read
            Scope sc(h, fine ? PF_CPAIR0 : PF_CPAIR, sizeof(T) * (4.0 * L.g.ncell + L.g.nvel), s,
                     1, 2.0 * fl);
            launch_cell_gs_pair<T>(L.g, C, buf[it & 1], buf[(it + 1) & 1], rhs, s);
        }
    }
    for (; it < nsweep; ++it)
        for (int par = 0; par < 2; ++par) {
            if (from_zero && it == 0 && par == 0) {   // red from zero: no neighbour terms
                Scope sc(h, PF_CFIRST, bytes_cell_first<T>(L.g), s, 1, 0.0);
                launch_cell_gs_colour<T>(L.g, C, par, phi, rhs, s, tpb_of<T>(h), true);
                continue;
            }
            Scope sc(h, fine ? PF_CSMOOTH0 : PF_CSMOOTH, bytes_cell_colour<T>(L.g), s, 1, fl);
            launch_cell_gs_colour<T>(L.g, C, par, phi, rhs, s, tpb_of<T>(h));
        }
}

// One velocity V-cycle for A phi = rhs with phi = 0 initially (App. C).
// Level l reads rhs (level 0: caller's vector) and writes phi.
template <typename T>
void vcycle_vel(stk_handle* h, int l, const T* rhs, T* phi, const MGParams& mp, cudaStream_t s) {
    const Level& L = h->lev[l];
    Work<T> W = work_of<T>(L);
    if (l >= lcoarse_of<T>(h)) {   // this level and all coarser ones in one launch
        Scope sc(h, PF_COARSE, 0.0, s);
        const size_t smi = coarse_smem_stk<T>(h, l, true);
        if (smi > 0) {
            const int nl = (int)h->lev.size();
            launch_coarse_stacked<T>(true, L.g.dim, h->nsl, clstk_of<T>(h) + (l - h->lstk), nl - h->lstk,
                                     nl - l, rhs, phi, mp.nu, mp.ncoarse, h->bulk, smi, s);
            return;
        }
        launch_coarse_vcycle_vel<T>(L.g.dim, L.g.nsl, clev_of<T>(h) + l, (int)h->lev.size() - l, rhs,
                                    phi, mp.nu, mp.ncoarse, h->bulk, coarse_smem<T>(h, l, true), s);
        return;
    }
    if (l >= lcluster_of<T>(h)) {  // this level down as one thread-block cluster
        Scope sc(h, PF_COARSE, 0.0, s);
        launch_cluster_vcycle_vel<T>(L.g.dim, L.g, clev_of<T>(h) + l, (int)h->lev.size() - l,
                                     lcoarse_of<T>(h) - l, rhs, phi, mp.nu, mp.ncoarse, h->bulk, s);
        return;
    }
    if (l >= lgrid_of<T>(h)) {     // this level down as one persistent multi-block launch
        Scope sc(h, PF_COARSE, 0.0, s);
        launch_grid_vcycle_vel<T>(L.g.dim, L.g, clev_of<T>(h) + l, (int)h->lev.size() - l,
                                  lcoarse_of<T>(h) - l, rhs, phi, mp.nu, mp.ncoarse, h->bulk, h->gbar,
                                  reinterpret_cast<const long long*>(h->gbar + 2), &h->gst->wait_status, s);
        return;
    }
    if (l + 1 == (int)h->lev.size() && smat_u_of<T>(L) && mp.ncoarse == SMAT_SWEEPS) {
        Scope sc(h, PF_COARSE, 0.0, s);
        launch_coarsest_apply<T>(L.g.nvel, smat_u_of<T>(L), rhs, phi, s);
        return;
    }
    // Below the finest level phi is a work array of this level whose wall
    // faces nothing ever writes (they stay the zeros it was allocated with),
    // and a first sweep from zero by colour kernels reads no unknown before
    // writing it: the zero fill is needed only at the finest level (the
    // caller's array), for two-colour sweeps (they read every value), with
    // bulk viscosity (full first sweep) or without sweeps.
    const int nsw = l + 1 == (int)h->lev.size() ? mp.ncoarse : mp.nu;
    if (l == 0 || l >= lpair_of<T>(h) || h->bulk || nsw < 1) launch_zero<T>(L.g.nvel, phi, s);
    if (l + 1 == (int)h->lev.size()) {
        vel_sweeps<T>(h, l, mp.ncoarse, phi, rhs, s, true);
        return;
    }
    const Level& Lc = h->lev[l + 1];
    Work<T> Wc = work_of<T>(Lc);
    vel_sweeps<T>(h, l, mp.nu, phi, rhs, s, true);
    {
        const bool st = sizeof(T) == 8 && l == 0;
        Scope sc(h, PF_VRES, bytes_vel_residual<T>(L.g), s, st ? stress_kernels(L.g) : 1);
        if (st)   // FP64 finest level: through the stresses
            launch_vel_residual_stress(L.g, h->lev[0].cd, h->sw, reinterpret_cast<const double*>(phi),
                                       reinterpret_cast<const double*>(rhs),
                                       reinterpret_cast<double*>(W.res_u), mp.nu > 0, s);
        else
            launch_vel_residual<T>(L.g, coef_of<T>(L), phi, rhs, W.res_u, s, mp.nu > 0);
    }
    {
        Scope sc(h, PF_VRESTR, sizeof(T) * (L.g.nvel + Lc.g.nvel), s);
        launch_vel_restrict<T>(L.g, W.res_u, Lc.g, Wc.rhs_u, s);
    }
    vcycle_vel<T>(h, l + 1, Wc.rhs_u, Wc.phi_u, mp, s);
    {
        Scope sc(h, PF_VPROL, sizeof(T) * (2.0 * L.g.nvel + Lc.g.nvel), s);
        launch_vel_prolong_add<T>(Lc.g, Wc.phi_u, L.g, phi, s);
    }
    vel_sweeps<T>(h, l, mp.nu, phi, rhs, s);
}

// One pressure V-cycle for L_rho phi = rhs with phi = 0 initially (App. C).
template <typename T>
void vcycle_cell(stk_handle* h, int l, const T* rhs, T* phi, const MGParams& mp, cudaStream_t s) {
    const Level& L = h->lev[l];
    Work<T> W = work_of<T>(L);
    if (l >= lcoarse_of<T>(h)) {
        Scope sc(h, PF_COARSE, 0.0, s);
        const size_t smi = coarse_smem_stk<T>(h, l, false);
        if (smi > 0) {
            const int nl = (int)h->lev.size();
            launch_coarse_stacked<T>(false, L.g.dim, h->nsl, clstk_of<T>(h) + (l - h->lstk), nl - h->lstk,
                                     nl - l, rhs, phi, mp.nu, mp.ncoarse, false, smi, s);
            return;
        }
        launch_coarse_vcycle_cell<T>(L.g.dim, L.g.nsl, clev_of<T>(h) + l, (int)h->lev.size() - l, rhs,
                                     phi, mp.nu, mp.ncoarse, coarse_smem<T>(h, l, false), s);
        return;
    }
    if (l >= lcluster_of<T>(h)) {
        Scope sc(h, PF_COARSE, 0.0, s);
        launch_cluster_vcycle_cell<T>(L.g.dim, L.g, clev_of<T>(h) + l, (int)h->lev.size() - l,
                                      lcoarse_of<T>(h) - l, rhs, phi, mp.nu, mp.ncoarse, s);
        return;
    }
    if (l >= lgrid_of<T>(h)) {
        Scope sc(h, PF_COARSE, 0.0, s);
        launch_grid_vcycle_cell<T>(L.g.dim, L.g, clev_of<T>(h) + l, (int)h->lev.size() - l,
                                   lcoarse_of<T>(h) - l, rhs, phi, mp.nu, mp.ncoarse, h->gbar,
                                   reinterpret_cast<const long long*>(h->gbar + 2), &h->gst->wait_status, s);
        return;
    }
    if (l + 1 == (int)h->lev.size() && smat_p_of<T>(L) && mp.ncoarse == SMAT_SWEEPS) {
        Scope sc(h, PF_COARSE, 0.0, s);
        launch_coarsest_apply<T>(L.g.ncell, smat_p_of<T>(L), rhs, phi, s);
        return;
    }
    // as for the velocity: the red cells from zero read no neighbour
    const int nsw = l + 1 == (int)h->lev.size() ? mp.ncoarse : mp.nu;
    if (l == 0 || l >= lpair_of<T>(h) || nsw < 1) launch_zero<T>(L.g.ncell, phi, s);
    if (l + 1 == (int)h->lev.size()) {
        cell_sweeps<T>(h, l, mp.ncoarse, phi, rhs, s, true);
        return;
    }
    const Level& Lc = h->lev[l + 1];
    Work<T> Wc = work_of<T>(Lc);
    cell_sweeps<T>(h, l, mp.nu, phi, rhs, s, true);
    {
        Scope sc(h, PF_CRES, sizeof(T) * (3.0 * L.g.ncell + L.g.nvel), s);
        launch_cell_residual<T>(L.g, coef_of<T>(L), phi, rhs, W.res_p, s, mp.nu > 0);
    }
    {
        Scope sc(h, PF_CRESTR, sizeof(T) * (L.g.ncell + Lc.g.ncell), s);
        launch_cell_restrict<T>(L.g, W.res_p, Lc.g, Wc.rhs_p, s);
    }
    vcycle_cell<T>(h, l + 1, Wc.rhs_p, Wc.phi_p, mp, s);
    {
        Scope sc(h, PF_CPROL, sizeof(T) * (2.0 * L.g.ncell + Lc.g.ncell), s);
        launch_cell_prolong_add<T>(Lc.g, Wc.phi_p, L.g, phi, s);
    }
    cell_sweeps<T>(h, l, mp.nu, phi, rhs, s);
}

// out[0] = sum x of a cell vector: FP32 vectors with 16-byte alignment
// take the wide-load reduction, the rest the plain one.  A stacked batch:
// the sum of each instance, instance y's at out[y * NDSC].
template <typename T>
void cell_sum(stk_handle* h, int n, const T* x, double* out, cudaStream_t s) {
    const int nsl = h->nsl;
    if constexpr (sizeof(T) == 4) {
        if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
            if (nsl > 1)
                launch_sum_f32x4_sl(n / nsl, nsl, reinterpret_cast<const float*>(x), h->red, out, NDSC, h->rcnt, s);
            else launch_sum_f32x4(n, reinterpret_cast<const float*>(x), h->red, out, h->rcnt, s);
            return;
        }
    }
    if (nsl > 1) launch_sum_sl<T>(n / nsl, nsl, x, h->red, out, NDSC, h->rcnt, s);
    else launch_sum<T>(n, x, h->red, out, h->rcnt, s);
}

// out = in - mean(in) (per instance of a stacked batch; sum from cell_sum)
template <typename T>
void sub_mean(stk_handle* h, int n, const T* in, T* out, double* sum, cudaStream_t s) {
    if (h->nsl > 1) launch_sub_mean_sl<T>(n / h->nsl, h->nsl, in, out, sum, NDSC, s);
    else if (in == out) launch_sub_mean<T>(n, out, sum, s);
    else launch_copy_sub_mean<T>(n, in, out, sum, s);
}

// phi = L~_rho^{-1} (r - mean r): the Poisson right-hand side is projected
// onto mean-zero vectors (the constant null space of L_rho, Sec. 3.2).
template <typename T>
void poisson_solve(stk_handle* h, const T* r, T* phi, const MGParams& mp, cudaStream_t s) {
    const Level& L = h->lev[0];
    Work<T> W = work_of<T>(L);
    PBuf<T>& B = pbuf_of<T>(h);
    const int nc = L.g.ncell;
    {
        Scope sc(h, PF_MEAN, 2.0 * sizeof(T) * nc, s, 2);
        cell_sum<T>(h, nc, r, h->dsc + DS_SUM, s);
        sub_mean<T>(h, nc, r, W.rhs_p, h->dsc + DS_SUM, s);
    }
    vcycle_cell<T>(h, 0, W.rhs_p, phi, mp, s);
    // further cycles: phi += V(r - L phi), the residual projected onto
    // mean-zero vectors like the right-hand side (Sec. 4.1.2)
    for (int c = 1; c < mp.cp; ++c) {
        {
            Scope sc(h, PF_CRES, sizeof(T) * (3.0 * nc + L.g.nvel), s);
            launch_cell_residual<T>(L.g, coef_of<T>(L), phi, W.rhs_p, B.rp, s);
        }
        {
            Scope sc(h, PF_MEAN, 3.0 * sizeof(T) * nc, s, 2);
            cell_sum<T>(h, nc, B.rp, h->dsc + DS_SUM + 4, s);
            sub_mean<T>(h, nc, B.rp, B.rp, h->dsc + DS_SUM + 4, s);
        }
        vcycle_cell<T>(h, 0, B.rp, B.dp, mp, s);
        { Scope sc(h, PF_ALG, 3.0 * sizeof(T) * nc, s); launch_axpy<T>(nc, T(1), B.dp, phi, s); }
    }
}

// Velocity subsolve: mp.cu V-cycles, the first from zero, each further one
// on the residual: x += V(r - A x) (Sec. 4.1.2).
template <typename T>
void velocity_solve(stk_handle* h, const T* r, T* x, const MGParams& mp, cudaStream_t s) {
    vcycle_vel<T>(h, 0, r, x, mp, s);
    const Level& L = h->lev[0];
    PBuf<T>& B = pbuf_of<T>(h);
    for (int c = 1; c < mp.cu; ++c) {
        {
            Scope sc(h, PF_VRES, bytes_vel_residual<T>(L.g), s);
            launch_vel_residual<T>(L.g, coef_of<T>(L), x, r, B.ru, s);
        }
        vcycle_vel<T>(h, 0, B.ru, B.du, mp, s);
        { Scope sc(h, PF_ALG, 3.0 * sizeof(T) * L.g.nvel, s); launch_axpy<T>(L.g.nvel, T(1), B.du, x, s); }
    }
}

template <typename T>
void remove_mean(stk_handle* h, T* x, cudaStream_t s) {
    const Level& L = h->lev[0];
    Scope sc(h, PF_MEAN, 3.0 * sizeof(T) * L.g.ncell, s, 2);
    cell_sum<T>(h, L.g.ncell, x, h->dsc + DS_SUM + 2, s);
    sub_mean<T>(h, L.g.ncell, x, x, h->dsc + DS_SUM + 2, s);
}

// x = P^{-1} b, Sec. 2.1-2.4; b, x packed Stokes vectors of precision T.
template <typename T>
void apply_precond(stk_handle* h, int which, const T* b, T* x, const MGParams& mp, cudaStream_t s) {
    const Level& L = h->lev[0];
    const Geom& g = L.g;
    Coef<T> C = coef_of<T>(L);
    Work<T> W = work_of<T>(L);
    PBuf<T>& B = pbuf_of<T>(h);
    const T* bu = b;
    const T* bp = b + g.nvel;
    T* xu = x;
    T* xp = x + g.nvel;
    const bool pois = h->theta != 0.0;
    const double alg_cell = sizeof(T) * 3.0 * g.ncell + sizeof(T) * g.nvel;
    switch (which) {
    case STK_P1: {
        velocity_solve<T>(h, bu, B.xs, mp, s);
        { Scope sc(h, PF_ALG, alg_cell, s); launch_div_plus<T>(g, B.xs, bp, B.bc, s); }
        poisson_solve<T>(h, B.bc, W.phi_p, mp, s);
        {
            Scope sc(h, PF_ALG, sizeof(T) * (3.0 * g.nvel + g.ncell), s);
            launch_sub_grad<T>(g, C.beta, B.xs, W.phi_p, xu, s);
        }
        { Scope sc(h, PF_ALG, alg_cell, s); launch_schur_combine<T>(g.ncell, h->dsc + DS_THETA, W.phi_p, C.mu2_c, C.lam_c, B.bc, xp, s); }
        break;
    }
    case STK_P2: {
        velocity_solve<T>(h, bu, xu, mp, s);
        { Scope sc(h, PF_ALG, alg_cell, s); launch_div_plus<T>(g, xu, bp, B.bc, s); }
        if (pois) poisson_solve<T>(h, B.bc, W.phi_p, mp, s);
        { Scope sc(h, PF_ALG, alg_cell, s); launch_schur_combine<T>(g.ncell, h->dsc + DS_THETA, pois ? W.phi_p : nullptr, C.mu2_c, C.lam_c, B.bc, xp, s); }
        break;
    }
    case STK_P3: {
        if (pois) poisson_solve<T>(h, bp, W.phi_p, mp, s);
        { Scope sc(h, PF_ALG, alg_cell, s); launch_schur_combine<T>(g.ncell, h->dsc + DS_THETA, pois ? W.phi_p : nullptr, C.mu2_c, C.lam_c, bp, xp, s); }
        {
            Scope sc(h, PF_ALG, sizeof(T) * (2.0 * g.nvel + g.ncell), s);
            launch_sub_grad<T>(g, (const T*)nullptr, bu, xp, B.tmpu, s);
        }
        velocity_solve<T>(h, B.tmpu, xu, mp, s);
        break;
    }
    case STK_P4: {
        velocity_solve<T>(h, bu, xu, mp, s);
        if (pois) poisson_solve<T>(h, bp, W.phi_p, mp, s);
        { Scope sc(h, PF_ALG, alg_cell, s); launch_schur_combine<T>(g.ncell, h->dsc + DS_THETA, pois ? W.phi_p : nullptr, C.mu2_c, C.lam_c, bp, xp, s); }
        break;
    }
    default: {  // STK_P5
        velocity_solve<T>(h, bu, B.xs, mp, s);
        { Scope sc(h, PF_ALG, alg_cell, s); launch_div_plus<T>(g, B.xs, bp, B.bc, s); }
        if (pois) poisson_solve<T>(h, B.bc, W.phi_p, mp, s);
        { Scope sc(h, PF_ALG, alg_cell, s); launch_schur_combine<T>(g.ncell, h->dsc + DS_THETA, pois ? W.phi_p : nullptr, C.mu2_c, C.lam_c, B.bc, xp, s); }
        {
            Scope sc(h, PF_ALG, bytes_vel_residual<T>(g), s);
            launch_vel_correction_rhs<T>(g, C, bu, xp, B.xs, B.tmpu, s);
        }
        velocity_solve<T>(h, B.tmpu, xu, mp, s);
        { Scope sc(h, PF_ALG, 3.0 * sizeof(T) * g.nvel, s); launch_axpy<T>(g.nvel, T(1), B.xs, xu, s); }
        break;
    }
    }
    remove_mean<T>(h, xp, s);
}

void clear_graphs(stk_handle* h) {
    if (h->graphs.empty() && h->cgraphs.empty() && h->pgraphs.empty()) return;
    cudaDeviceSynchronize();   // no launch of these graphs may still be in flight
    for (auto& kv : h->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        for (auto& r : kv.second.recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
    }
    h->graphs.clear();
    // the GMRES cycle and phase graphs contain preconditioner applications
    for (auto& kv : h->cgraphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    h->cgraphs.clear();
    for (auto& kv : h->pgraphs)
        if (kv.second.first) cudaGraphExecDestroy(kv.second.first);
    h->pgraphs.clear();
}

// x = P^{-1} b through a CUDA graph captured on first use (one graph per
// preconditioner, precision and buffer pair), so that the ~10^2 kernels of
// the V-cycles are submitted with one launch.
template <typename T>
int run_precond(stk_handle* h, int which, const T* b, T* x, const MGParams& mp, cudaStream_t s) {
    if (!h->use_graphs) {
        apply_precond<T>(h, which, b, x, mp, s);
        CKL();
        return STK_OK;
    }
    auto key = std::make_tuple(which, (int)sizeof(T), (const void*)b, (void*)x, mp.nu, mp.ncoarse,
                               mp.cu * 1000 + mp.cp, h->prof ? 1 : 0);
    auto it = h->graphs.find(key);
    if (it == h->graphs.end()) {
        stk_handle::GraphEntry e;
        CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        h->capturing = true;
        h->cap_kernels = 0;
        h->caprecs.clear();
        apply_precond<T>(h, which, b, x, mp, h->cap);
        h->capturing = false;
        cudaGraph_t g = nullptr;
        cudaError_t ec = cudaStreamEndCapture(h->cap, &g);
        if (ec != cudaSuccess) return fail(h, STK_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ec));
        ec = cudaGraphInstantiate(&e.exec, g, 0);
        cudaGraphDestroy(g);
        if (ec != cudaSuccess) return fail(h, STK_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ec));
        e.kernels = h->cap_kernels;
        e.recs = h->caprecs;
        h->caprecs.clear();
        it = h->graphs.emplace(key, std::move(e)).first;
    }
    CK(cudaGraphLaunch(it->second.exec, s));
    h->nkern += it->second.kernels;
    if (h->prof) {   // read the graph's event pairs before its next launch
        h->recs.insert(h->recs.end(), it->second.recs.begin(), it->second.recs.end());
        prof_flush(h);
    }
    return STK_OK;
}

double scalar_vcycles(const stk_handle* h, int which, const MGParams& mp) {
    const double u = double(h->dim) * mp.cu;          // d scalar cycles per velocity cycle
    const double p = h->theta != 0.0 ? mp.cp : 0.0;
    if (which == STK_P1) return u + mp.cp;
    if (which == STK_P5) return 2.0 * u + p;
    return u + p;
}

int nstokes(const stk_handle* h) { return h->lev[0].g.nvel + h->lev[0].g.ncell; }

int check_ptrs(stk_handle* h, const void* const* u, const void* p) {
    if (!u || !p) return fail(h, STK_ERR_ARG, "null array pointer");
    for (int a = 0; a < h->dim; ++a)
        if (!u[a]) return fail(h, STK_ERR_ARG, "null face array %d", a);
    return STK_OK;
}

// gather caller's face/cell arrays into a packed vector and back
int gather(stk_handle* h, const double* const* u, const double* p, double* packed, cudaStream_t s) {
    const Geom& g = h->lev[0].g;
    for (int a = 0; a < g.dim; ++a)
        CK(cudaMemcpyAsync(packed + g.foff[a], u[a], sizeof(double) * g.fsize[a],
                           cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(packed + g.nvel, p, sizeof(double) * g.ncell, cudaMemcpyDeviceToDevice, s));
    return STK_OK;
}

int scatter(stk_handle* h, const double* packed, double* const* u, double* p, cudaStream_t s) {
    const Geom& g = h->lev[0].g;
    for (int a = 0; a < g.dim; ++a)
        CK(cudaMemcpyAsync(u[a], packed + g.foff[a], sizeof(double) * g.fsize[a],
                           cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(p, packed + g.nvel, sizeof(double) * g.ncell, cudaMemcpyDeviceToDevice, s));
    return STK_OK;
}

int ensure_krylov(stk_handle* h, int m) {
    if (m <= h->m_alloc) return STK_OK;
    const int n = nstokes(h);
    for (int i = (int)h->V.size(); i < m + 1; ++i) {
        double* v;
        CK(dalloc(h, &v, n));
        h->V.push_back(v);
    }
    for (int i = (int)h->Z.size(); i < m; ++i) {
        float* z;
        CK(dalloc(h, &z, n));
        h->Z.push_back(z);
    }
    h->m_alloc = m;
    return STK_OK;
}

// ---------------------------------------------------------------- GMRES core
// The Arnoldi process of Sec. 3.2 with its least-squares problem kept on the
// device (gmres.cu): one GMRES cycle is enqueued as phases -- the true
// residual and the stopping test, the first basis vector, Arnoldi steps
// 0..m-1, the update of x -- each gated by a decision a kernel of the
// previous phase wrote.  Inside a CUDA graph the gates are conditional
// nodes, so a whole cycle is one graph launch and the host reads the state
// once per cycle; without graphs (profiling) the host reads each decision.

// Orthogonalise w = V[j+1] against V[0..j] by modified Gram-Schmidt:
// h_0 = <w, v_0>; for k = 0..j: w -= h_k v_k fused with h_{k+1} = <w, v_{k+1}>
// (the last step forms ||w||^2 in DS_N2 instead).  The coefficients stay in
// device memory (DS_H) for the Givens kernel.
// A stacked batch runs the same steps per instance (instance y's scalars
// at y * NDSC), bitwise as each instance alone.
void orth_enqueue(stk_handle* h, int j, cudaStream_t s) {
    const int n = nstokes(h);
    const bool sl = h->nsl > 1;
    double* w = h->V[j + 1];
    double* hd = h->dsc + DS_H;
    {
        Scope sc(h, PF_MDOT, 16.0 * n, s, 1);
        const double* v0 = h->V[0];
        if (sl) launch_multidot_sl(h->smap, h->nsl, 0, &v0, w, h->red, hd, NDSC, h->rcnt, s);
        else launch_multidot(n, 0, &v0, w, h->red, hd, h->rcnt, s);
    }
    for (int k = 0; k <= j; ++k) {
        const bool last = k == j;
        Scope sc(h, PF_UPD, 8.0 * n * (last ? 3 : 4), s, 1);
        double* out = last ? h->dsc + DS_N2 : hd + k + 1;
        if (sl)
            launch_mgs_step_sl(h->smap, h->nsl, h->V[k], last ? nullptr : h->V[k + 1], hd, NDSC, k, w,
                               h->red, out, NDSC, h->rcnt, s);
        else
            launch_mgs_step(n, h->V[k], last ? nullptr : h->V[k + 1], hd, k, w, h->red, out, h->rcnt, s);
    }
}

// out[0] = ||x||^2 (device; per instance of a stacked batch at stride NDSC)
void norm_enqueue(stk_handle* h, const double* x, double* out, cudaStream_t s) {
    const int n = nstokes(h);
    Scope sc(h, PF_MDOT, 8.0 * n, s, 1);
    if (h->nsl > 1) launch_multidot_sl(h->smap, h->nsl, -1, nullptr, x, h->red, out, NDSC, h->rcnt, s);
    else launch_multidot(n, -1, nullptr, x, h->red, out, h->rcnt, s);
}

struct CycleCtx {
    stk_handle* h;
    int which, m;
    bool flex;
    MGParams mp;
};

// x = P^{-1} b inside a GMRES phase: captured kernel by kernel into a cycle
// graph, otherwise as the preconditioner's own graph (run_precond)
template <typename T>
int precond_enqueue(stk_handle* h, int which, const T* b, T* x, const MGParams& mp, cudaStream_t s) {
    if (h->capturing) {
        apply_precond<T>(h, which, b, x, mp, s);
        return STK_OK;
    }
    return run_precond<T>(h, which, b, x, mp, s);
}

// phase 1: r = b - M x, ||r||^2, stopping test (gate of phase 2)
void enq_check(const CycleCtx& c, cudaStream_t s, cudaGraphConditionalHandle hpre, int use) {
    stk_handle* h = c.h;
    const Geom& g = h->lev[0].g;
    {
        Scope sc(h, PF_MATVEC, bytes_matvec(g, 8) + 8.0 * nstokes(h), s, stress_kernels(g));
        launch_stokes_matvec_stress(g, h->lev[0].cd, h->sw, h->xk, h->bk, h->tmp, s);
    }
    norm_enqueue(h, h->tmp, h->dsc + DS_N2 + 1, s);
    {
        Scope sc(h, PF_ALG, 0.0, s);
        launch_gm_check(h->gst, h->nsl, h->gcond, h->dsc + DS_N2 + 1, NDSC, hpre, use, s);
    }
}

// phase 2: v_0 = P^{-1} r (left) or r (flexible), beta, target (gates of the
// first Arnoldi step and of the update)
int enq_pre(const CycleCtx& c, cudaStream_t s, cudaGraphConditionalHandle h0,
            cudaGraphConditionalHandle hfin, int use) {
    stk_handle* h = c.h;
    if (c.flex) {
        CK(cudaMemcpyAsync(h->V[0], h->tmp, sizeof(double) * nstokes(h), cudaMemcpyDeviceToDevice, s));
    } else {
        int rc = precond_enqueue<double>(h, c.which, h->tmp, h->V[0], c.mp, s);
        if (rc) return rc;
        norm_enqueue(h, h->V[0], h->dsc + DS_N2 + 2, s);
    }
    {
        Scope sc(h, PF_ALG, 0.0, s);
        launch_gm_start(h->gst, h->nsl, h->gcond, h->dsc + DS_N2 + 2, NDSC, h0, use, hfin, use, s);
    }
    return STK_OK;
}

// phase 3 + j: Arnoldi step j (gate of step j + 1)
int enq_step(const CycleCtx& c, int j, cudaStream_t s, cudaGraphConditionalHandle hn, int use) {
    stk_handle* h = c.h;
    const Geom& g = h->lev[0].g;
    const int n = nstokes(h);
    {   // v_j /= beta (j = 0) or h_{j,j-1}
        Scope sc(h, PF_COMB, 16.0 * n, s);
        if (h->nsl > 1) launch_scale_dev_sl(h->smap, h->nsl, h->V[j], h->gst, j, s);
        else launch_scale_dev(n, h->V[j], &h->gst->inv_scale, s);
    }
    if (c.flex) {
        {
            Scope sc(h, PF_CONV, 12.0 * n, s);
            launch_convert<double, float>(n, h->V[j], h->pf.in, s);
        }
        int rc = precond_enqueue<float>(h, c.which, h->pf.in, h->Z[j], c.mp, s);
        if (rc) return rc;
        {   // the FP64 matvec of the FP32 direction z_j (converted once)
            Scope sc(h, PF_CONV, 12.0 * n, s);
            launch_convert<float, double>(n, h->Z[j], h->tmp, s);
        }
        Scope sc(h, PF_MATVEC, bytes_matvec(g, 8), s, stress_kernels(g));
        launch_stokes_matvec_stress(g, h->lev[0].cd, h->sw, h->tmp, nullptr, h->V[j + 1], s);
    } else {
        {
            Scope sc(h, PF_MATVEC, bytes_matvec(g, 8), s, stress_kernels(g));
            launch_stokes_matvec_stress(g, h->lev[0].cd, h->sw, h->V[j], nullptr, h->tmp, s);
        }
        int rc = precond_enqueue<double>(h, c.which, h->tmp, h->V[j + 1], c.mp, s);
        if (rc) return rc;
    }
    orth_enqueue(h, j, s);
    Scope sc(h, PF_ALG, 0.0, s);
    launch_gm_step(h->gst, h->nsl, h->gcond, j, h->dsc + DS_H, h->dsc + DS_N2, NDSC, hn, use, s);
    return STK_OK;
}

// last phase: y = R^{-1} g, x += V y (left) or Z y (flexible)
void enq_fin(const CycleCtx& c, cudaStream_t s) {
    stk_handle* h = c.h;
    const int n = nstokes(h);
    { Scope sc(h, PF_ALG, 0.0, s); launch_gm_finish(h->gst, h->nsl, s); }
    Scope sc(h, PF_COMB, (c.flex ? 4.0 : 8.0) * n * c.m + 16.0 * n, s);
    const bool sl = h->nsl > 1;
    if (c.flex) {
        std::vector<const float*> Zp(h->Z.begin(), h->Z.begin() + c.m);
        if (sl) launch_combine_dev_sl<float>(h->smap, h->nsl, c.m, Zp.data(), h->gst, h->xk, s);
        else launch_combine_dev<float>(n, c.m, Zp.data(), h->gst->y, &h->gst->k, h->xk, s);
    } else {
        std::vector<const double*> Vp(h->V.begin(), h->V.begin() + c.m);
        if (sl) launch_combine_dev_sl<double>(h->smap, h->nsl, c.m, Vp.data(), h->gst, h->xk, s);
        else launch_combine_dev<double>(n, c.m, Vp.data(), h->gst->y, &h->gst->k, h->xk, s);
    }
}

// Append the chain of one instance's GMRES cycle to the graph G: conditional
// (if) nodes, each holding one phase captured from the enqueue functions
// above.  The first node's condition is 1 at every launch; its gate kernel
// opens the stopping test only while the instance is still running, and each
// later condition is set by the kernels of the phase before it.
int build_chain(cudaGraph_t G, const CycleCtx& c, stk_handle::CycleGraph& out) {
    stk_handle* h = c.h;
    const int m = c.m;
    std::vector<cudaGraphConditionalHandle> hs(m + 4);   // gate, check, pre, fin, step 0..m-1
    int rc = STK_OK;
    for (int i = 0; i < m + 4 && rc == STK_OK; ++i) {
        cudaError_t e = cudaGraphConditionalHandleCreate(&hs[i], G, i == 0 ? 1u : 0u,
                                                         cudaGraphCondAssignDefault);
        if (e != cudaSuccess) rc = fail(h, STK_ERR_CUDA, "conditional handle: %s", cudaGetErrorString(e));
    }
    const cudaGraphConditionalHandle hgate = hs[0], hchk = hs[1], hpre = hs[2], hfin = hs[3];
    auto hstep = [&](int j) { return hs[4 + j]; };
    cudaGraphNode_t prev = nullptr;
    // add an if-node after prev whose body is captured from fn(stream)
    auto add_if = [&](cudaGraphConditionalHandle hc, auto&& fn, long long& kernels) -> int {
        if (rc) return rc;
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = hc;
        np.conditional.type = cudaGraphCondTypeIf;
        np.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        cudaError_t e = cudaGraphAddNode(&node, G, prev ? &prev : nullptr, nullptr, prev ? 1 : 0, &np);
        if (e != cudaSuccess) return rc = fail(h, STK_ERR_CUDA, "conditional node: %s", cudaGetErrorString(e));
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(h->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return rc = fail(h, STK_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
        h->capturing = true;
        h->cap_kernels = 0;
        int frc = fn(h->cap);
        h->capturing = false;
        cudaGraph_t got = nullptr;
        e = cudaStreamEndCapture(h->cap, &got);
        if (frc) return rc = frc;
        if (e != cudaSuccess) return rc = fail(h, STK_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
        kernels = h->cap_kernels;
        prev = node;
        return STK_OK;
    };
    out.k_step.assign(m, 0);
    add_if(hgate, [&](cudaStream_t s) {
        Scope sc(h, PF_ALG, 0.0, s);
        launch_gm_gate(h->gst, h->nsl, h->gcond, hchk, s);
        return STK_OK;
    }, out.k_gate);
    add_if(hchk, [&](cudaStream_t s) { enq_check(c, s, hpre, 1); return STK_OK; }, out.k_chk);
    add_if(hpre, [&](cudaStream_t s) { return enq_pre(c, s, hstep(0), hfin, 1); }, out.k_pre);
    for (int j = 0; j < m; ++j)
        add_if(hstep(j), [&](cudaStream_t s) {
            return enq_step(c, j, s, j + 1 < m ? hstep(j + 1) : 0, j + 1 < m ? 1 : 0);
        }, out.k_step[j]);
    add_if(hfin, [&](cudaStream_t s) { enq_fin(c, s); return STK_OK; }, out.k_fin);
    return rc;
}

int instantiate(stk_handle* h, cudaGraph_t G, cudaGraphExec_t* exec) {
    cudaError_t e = cudaGraphInstantiate(exec, G, 0);
    if (e != cudaSuccess) {
        *exec = nullptr;
        cudaGetLastError();
        return fail(h, STK_ERR_CUDA, "cycle graph instantiate: %s", cudaGetErrorString(e));
    }
    return STK_OK;
}

// The graph of one GMRES cycle of one instance.
int build_cycle_graph(const CycleCtx& c, stk_handle::CycleGraph& out) {
    stk_handle* h = c.h;
    cudaGraph_t G = nullptr;
    CK(cudaGraphCreate(&G, 0));
    int rc = build_chain(G, c, out);
    if (rc == STK_OK) rc = instantiate(h, G, &out.exec);
    cudaGraphDestroy(G);
    cudaGetLastError();
    return rc;
}

// One phase of a host-gated cycle: 0 the stopping test, 1 the first basis
// vector, 2 + j Arnoldi step j, m + 2 the update of x.
int enq_phase(const CycleCtx& c, int ph, cudaStream_t s) {
    if (ph == 0) {
        enq_check(c, s, 0, 0);
        return STK_OK;
    }
    if (ph == 1) return enq_pre(c, s, 0, 0, 0);
    if (ph < c.m + 2) return enq_step(c, ph - 2, s, 0, 0);
    enq_fin(c, s);
    return STK_OK;
}

// Run phase ph on stream s: one launch of a graph of that phase (captured on
// first use), or kernel by kernel when graphs are off or profiling is on.
int run_phase(const CycleCtx& c, int ph, cudaStream_t s) {
    stk_handle* h = c.h;
    if (!h->use_graphs || h->prof) {
        int rc = enq_phase(c, ph, s);
        if (rc) return rc;
        CKL();
        return STK_OK;
    }
    auto key = std::make_tuple(ph, c.which, c.flex ? 1 : 0, c.m, c.mp.nu, c.mp.ncoarse,
                               c.mp.cu * 1000 + c.mp.cp);
    auto f = h->pgraphs.find(key);
    if (f == h->pgraphs.end()) {
        CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        h->capturing = true;
        h->cap_kernels = 0;
        int rc = enq_phase(c, ph, h->cap);
        h->capturing = false;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->cap, &g);
        if (rc) return rc;
        if (e != cudaSuccess) return fail(h, STK_ERR_CUDA, "phase capture: %s", cudaGetErrorString(e));
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(h, STK_ERR_CUDA, "phase graph instantiate: %s", cudaGetErrorString(e));
        f = h->pgraphs.emplace(key, std::make_pair(ex, h->cap_kernels)).first;
    }
    CK(cudaGraphLaunch(f->second.first, s));
    h->nkern += f->second.second;
    return STK_OK;
}

// One GMRES instance advanced in lockstep with others (Sec. 3.2, Sec. 4).
// A stacked batch is one instance here: its records advance together, each
// on its own (the device kernels skip an instance's record where its phase
// is not open).
struct Inst {
    stk_handle* h = nullptr;
    cudaStream_t s = nullptr;
    stk_solve_info info{};
    int rc = STK_OK;
    bool done = false;              // solve finished (converged, maxit or error)
    stk_handle::CycleGraph* cg = nullptr;
};

constexpr size_t GM_HEADER = offsetof(GmState, H);   // bytes the host reads per cycle

int sync_all(std::vector<Inst*>& v) {
    int rc = STK_OK;
    for (Inst* it : v) {
        cudaError_t e = cudaStreamSynchronize(it->s);
        if (e != cudaSuccess && it->rc == STK_OK) {
            it->rc = fail(it->h, STK_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
            it->done = true;
            rc = it->rc;
        }
        e = cudaGetLastError();
        if (e != cudaSuccess && it->rc == STK_OK) {
            it->rc = fail(it->h, STK_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
            it->done = true;
            rc = it->rc;
        }
    }
    return rc;
}

void finish(Inst* it, int rc) {
    if (it->rc == STK_OK) it->rc = rc;
    it->done = true;
}

// the group decisions and every instance's record header
void read_header(Inst* it) {
    stk_handle* h = it->h;
    cudaMemcpyAsync(h->gcond_host, h->gcond, sizeof(unsigned) * GM_NCOND, cudaMemcpyDeviceToHost, it->s);
    if (h->nsl == 1)
        cudaMemcpyAsync(h->gst_host, h->gst, GM_HEADER, cudaMemcpyDeviceToHost, it->s);
    else
        cudaMemcpy2DAsync(h->gst_host, sizeof(GmState), h->gst, sizeof(GmState), GM_HEADER, h->nsl,
                          cudaMemcpyDeviceToHost, it->s);
}

// Summarise the instances' records into the info record; finish the solve
// once no instance is running (the first failing instance, in order, gives
// the error).
void settle(Inst* it) {
    stk_handle* h = it->h;
    bool running = false, all_conv = true;
    stk_solve_info& a = it->info;
    a.iterations = a.restarts = 0;
    a.true_residual = a.est_residual = a.scalar_vcycles = 0.0;
    int bad = -1, bad_state = GM_CONVERGED;
    for (int y = 0; y < h->nsl; ++y) {
        const GmState& st = h->gst_host[y];
        const stk_solve_info& f = h->sinfo[y];
        running = running || st.state == GM_RUNNING;
        all_conv = all_conv && st.state == GM_CONVERGED;
        a.iterations = std::max(a.iterations, f.iterations);
        a.restarts = std::max(a.restarts, f.restarts);
        a.true_residual = std::max(a.true_residual, f.true_residual);
        a.est_residual = std::max(a.est_residual, f.est_residual);
        a.scalar_vcycles = std::max(a.scalar_vcycles, f.scalar_vcycles);
        if (bad < 0 && st.state != GM_RUNNING && st.state != GM_CONVERGED && st.state != GM_MAXIT) {
            bad = y;
            bad_state = st.state;
        }
    }
    if (running) return;
    a.converged = all_conv ? 1 : 0;
    if (all_conv) { finish(it, STK_OK); return; }
    char who[32] = "";
    if (h->nsl > 1) snprintf(who, sizeof who, "instance %d: ", bad < 0 ? 0 : bad);
    if (bad < 0) { finish(it, STK_ERR_NOT_CONVERGED); return; }
    if (bad_state == GM_TIMEOUT) {
        finish(it, fail(h, STK_ERR_TIMEOUT, "%sa bounded device wait (grid barrier) ran out", who));
        return;
    }
    static const char* why[] = {"", "non-finite right-hand side", "non-finite residual",
                                "non-finite preconditioned residual",
                                "non-finite value in the Arnoldi process", "non-finite GMRES update"};
    const int w = h->gst_host[bad].why;
    finish(it, fail(h, STK_ERR_NONFINITE, "%s%s", who, why[w >= 1 && w <= 5 ? w : 0]));
}

// Fold the records read after a cycle into the per-instance info records.
void absorb_cycle(Inst* it, const stk_solver_params& prm, const MGParams& mp) {
    stk_handle* h = it->h;
    const unsigned* gc = h->gcond_host;
    const double sv = scalar_vcycles(h, prm.precond, mp);
    int steps_max = 0;
    for (int y = 0; y < h->nsl; ++y) {
        const GmState& st = h->gst_host[y];
        stk_solve_info& f = h->sinfo[y];
        const int steps = st.iterations - h->sit_before[y];
        steps_max = std::max(steps_max, steps);
        f.scalar_vcycles += sv * steps + ((prm.precision != STK_MIXED && st.cond[GM_COND_PRE]) ? sv : 0.0);
        f.iterations = st.iterations;
        f.restarts = st.restarts;
        f.true_residual = st.bnorm > 0.0 ? st.rnorm / st.bnorm : 0.0;
        f.est_residual = st.bnorm > 0.0 ? st.est / st.bnorm : 0.0;
        f.converged = st.state == GM_CONVERGED ? 1 : 0;
        h->sit_before[y] = st.iterations;
    }
    if (it->cg) {   // kernels the graph ran: the gates the device opened
        const auto& cg = *it->cg;
        h->nkern += cg.k_gate + (gc[GM_COND_CHK] ? cg.k_chk : 0) + (gc[GM_COND_PRE] ? cg.k_pre : 0) +
                    (gc[GM_COND_FIN] ? cg.k_fin : 0);
        for (int j = 0; j < steps_max && j < (int)cg.k_step.size(); ++j) h->nkern += cg.k_step[j];
    }
    settle(it);
}

// zero the part of the packed vector x that belongs to instance y
void zero_instance(stk_handle* h, double* x, int y, cudaStream_t s) {
    if (h->nsl == 1) {
        cudaMemsetAsync(x, 0, sizeof(double) * nstokes(h), s);
        return;
    }
    const SliceMap& m = h->smap;
    for (int k = 0; k < 3; ++k)
        cudaMemsetAsync(x + m.off[k] + (size_t)y * m.len[k], 0, sizeof(double) * m.len[k], s);
}

// Restarted GMRES for every instance: left-preconditioned with an FP64
// preconditioner, or flexible with an FP32 preconditioner (precision MIXED).
// Stopping rule: ||b - M x|| <= rtol ||b||, checked at the start of every
// cycle; inside a cycle the Arnoldi estimate must fall to rtol ||b||
// (flexible) or to its start value times rtol ||b|| / ||b - M x|| (left).
// With cycle_graphs (a single solve or a small batch, graphs on, profiling
// off) each cycle of each instance is one graph launch and the host waits
// once per cycle and instance, each instance at its own pace; otherwise the
// host gates the phases of all instances together, one synchronisation per
// phase for the whole batch, each phase one graph launch.
void gmres_lockstep(std::vector<Inst>& insts, const stk_solver_params& prm, bool cycle_graphs) {
    const int m = prm.restart;
    const bool flex = prm.precision == STK_MIXED;
    MGParams mp;
    mp.nu = prm.nu;
    mp.ncoarse = prm.ncoarse;
    mp.cu = prm.vcycles_u;
    mp.cp = prm.vcycles_p;
    std::vector<Inst*> act;
    for (auto& it : insts) {
        if (it.done) continue;
        int rc = ensure_krylov(it.h, m);
        if (rc) { finish(&it, rc); continue; }
        stk_handle* h = it.h;
        h->sinfo.assign(h->nsl, stk_solve_info{});
        h->sit_before.assign(h->nsl, 0);
        norm_enqueue(h, h->bk, h->dsc + DS_N2 + 3, it.s);
        launch_gm_begin(h->gst, h->nsl, h->gcond, h->dsc + DS_N2 + 3, NDSC, prm.rtol, prm.maxit, m,
                        flex ? 1 : 0, it.s);
        ++h->nkern;
        read_header(&it);
        act.push_back(&it);
    }
    sync_all(act);
    for (Inst* it : act) {
        if (it->done) continue;
        stk_handle* h = it->h;
        for (int y = 0; y < h->nsl; ++y) {
            const GmState& st = h->gst_host[y];
            if (st.state == GM_CONVERGED) {   // zero right-hand side: x = 0
                zero_instance(h, h->xk, y, it->s);
                h->sinfo[y].converged = 1;
            }
        }
        settle(it);
    }
    // graphs of the cycle (built on first use per handle and configuration)
    for (Inst* it : act) {
        if (it->done || !cycle_graphs) continue;
        stk_handle* h = it->h;
        it->cg = nullptr;
        if (!h->use_graphs || h->prof) continue;
        auto key = std::make_tuple(prm.precond, flex ? 1 : 0, m, mp.nu, mp.ncoarse, mp.cu * 1000 + mp.cp);
        auto f = h->cgraphs.find(key);
        if (f == h->cgraphs.end()) {
            stk_handle::CycleGraph cg;
            CycleCtx c{h, prm.precond, m, flex, mp};
            if (build_cycle_graph(c, cg) != STK_OK) {
                h->use_graphs = false;   // fall back to host-gated phases
                continue;
            }
            f = h->cgraphs.emplace(key, std::move(cg)).first;
        }
        it->cg = &f->second;
    }
    auto open_ = [](Inst* it, int slot) { return it->h->gcond_host[slot] != 0; };
    bool all_graphs = cycle_graphs;
    for (auto& it : insts)
        if (!it.done && !it.cg) all_graphs = false;
    if (all_graphs) {
        // Every instance advances on its own: a cycle graph launch, the read
        // of its records and an event; the host polls the events and starts
        // an instance's next cycle as soon as its last one has ended, so a
        // small instance never waits for a large one.
        auto launch = [](Inst* it) {
            cudaError_t e = cudaGraphLaunch(it->cg->exec, it->s);
            if (e != cudaSuccess) {
                finish(it, fail(it->h, STK_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e)));
                return;
            }
            read_header(it);
            cudaEventRecord(it->h->cyc, it->s);
        };
        std::vector<Inst*> pending;
        for (auto& it : insts)
            if (!it.done) {
                launch(&it);
                if (!it.done) pending.push_back(&it);
            }
        Nvtx range("gmres cycles");
        while (!pending.empty()) {
            bool moved = false;
            for (size_t i = 0; i < pending.size();) {
                Inst* it = pending[i];
                const cudaError_t q = cudaEventQuery(it->h->cyc);
                if (q == cudaErrorNotReady) {
                    ++i;
                    continue;
                }
                moved = true;
                if (q != cudaSuccess) {
                    finish(it, fail(it->h, STK_ERR_CUDA, "cycle: %s", cudaGetErrorString(q)));
                } else {
                    absorb_cycle(it, prm, mp);
                    if (!it->done) launch(it);
                }
                if (it->done) {
                    pending[i] = pending.back();
                    pending.pop_back();
                } else {
                    ++i;
                }
            }
            if (!moved) std::this_thread::yield();
        }
    }
    while (!all_graphs) {
        act.clear();
        for (auto& it : insts)
            if (!it.done) act.push_back(&it);
        if (act.empty()) break;
        Nvtx range("gmres cycle");
        std::vector<Inst*> eager;
        for (Inst* it : act) {
            if (it->cg) {
                cudaError_t e = cudaGraphLaunch(it->cg->exec, it->s);
                if (e != cudaSuccess) { finish(it, fail(it->h, STK_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e))); continue; }
                read_header(it);
            } else {
                eager.push_back(it);
            }
        }
        if (!eager.empty()) {   // the same phases, gated by the host
            for (Inst* it : eager) {
                CycleCtx c{it->h, prm.precond, m, flex, mp};
                int rc = run_phase(c, 0, it->s);
                if (rc) { finish(it, rc); continue; }
                read_header(it);
            }
            sync_all(eager);
            std::vector<Inst*> run;
            for (Inst* it : eager)
                if (!it->done && open_(it, GM_COND_PRE)) run.push_back(it);
            for (Inst* it : run) {
                CycleCtx c{it->h, prm.precond, m, flex, mp};
                int rc = run_phase(c, 1, it->s);
                if (rc) { finish(it, rc); continue; }
                read_header(it);
            }
            sync_all(run);
            for (int j = 0; j < m; ++j) {
                std::vector<Inst*> step;
                for (Inst* it : run)
                    if (!it->done && open_(it, GM_COND_STEP0 + j)) step.push_back(it);
                if (step.empty()) break;
                for (Inst* it : step) {
                    CycleCtx c{it->h, prm.precond, m, flex, mp};
                    int rc = run_phase(c, 2 + j, it->s);
                    if (rc) { finish(it, rc); continue; }
                    read_header(it);
                }
                sync_all(step);
            }
            for (Inst* it : run) {
                if (it->done || !open_(it, GM_COND_FIN)) continue;
                CycleCtx c{it->h, prm.precond, m, flex, mp};
                int rc = run_phase(c, m + 2, it->s);
                if (rc) { finish(it, rc); continue; }
                read_header(it);
            }
        }
        sync_all(act);
        for (Inst* it : act)
            if (!it->done) absorb_cycle(it, prm, mp);
    }
    std::vector<Inst*> all;
    for (auto& it : insts) all.push_back(&it);
    // residual histories of the solve
    for (Inst* it : all) {
        stk_handle* h = it->h;
        cudaMemcpyAsync(h->gst_host, h->gst, sizeof(GmState) * h->nsl, cudaMemcpyDeviceToHost, it->s);
    }
    sync_all(all);
    for (Inst* it : all) {
        stk_handle* h = it->h;
        h->hist_true.assign(h->nsl, {});
        h->hist_est.assign(h->nsl, {});
        for (int y = 0; y < h->nsl; ++y) {
            const GmState& st = h->gst_host[y];
            h->hist_true[y].assign(st.hist, st.hist + std::min(st.nhist, GM_NHIST));
            h->hist_est[y].assign(st.est_hist, st.est_hist + std::min(st.nest, GM_NEST));
        }
    }
}

int validate_params(stk_handle* h, const stk_solver_params& prm) {
    if (prm.precond < STK_P1 || prm.precond > STK_P5) return fail(h, STK_ERR_ARG, "preconditioner must be 1..5");
    if (prm.restart < 1 || prm.restart > 32) return fail(h, STK_ERR_ARG, "restart must be 1..32");
    if (!(prm.rtol > 0.0)) return fail(h, STK_ERR_ARG, "rtol must be > 0");
    if (prm.maxit < 1) return fail(h, STK_ERR_ARG, "maxit must be >= 1");
    if (prm.precision != STK_FP64 && prm.precision != STK_MIXED) return fail(h, STK_ERR_ARG, "bad precision");
    if (prm.nu < 0 || prm.ncoarse < 1) return fail(h, STK_ERR_ARG, "bad sweep counts");
    if (prm.vcycles_u < 1 || prm.vcycles_u > 64 || prm.vcycles_p < 1 || prm.vcycles_p > 64)
        return fail(h, STK_ERR_ARG, "V-cycles per subsolve must be 1..64");
    return STK_OK;
}

bool is_pow2(int v) { return v >= 2 && (v & (v - 1)) == 0; }

// level descriptors of the single-block coarse-level kernel (they embed the
// coefficient pointers, so they are rewritten when the bulk term toggles)
cudaError_t upload_clevels(stk_handle* h) {
    const int nl = (int)h->lev.size();
    std::vector<CLevel<double>> cd(nl);
    std::vector<CLevel<float>> cf(nl);
    for (int l = 0; l < nl; ++l) {
        const Level& L = h->lev[l];
        cd[l] = CLevel<double>{L.g, L.cd, L.wd.phi_u, L.wd.rhs_u, L.wd.res_u, L.wd.phi_p, L.wd.rhs_p, L.wd.res_p};
        cf[l] = CLevel<float>{L.g, L.cf, L.wf.phi_u, L.wf.rhs_u, L.wf.res_u, L.wf.phi_p, L.wf.rhs_p, L.wf.res_p};
        cd[l].smat_u = L.smat_ud;
        cd[l].smat_p = L.smat_pd;
        cf[l].smat_u = L.smat_uf;
        cf[l].smat_p = L.smat_pf;
        cd[l].smat_nc = cf[l].smat_nc = (L.smat_ud || L.smat_pd) ? SMAT_SWEEPS : 0;
    }
    cudaError_t e = cudaMemcpy(h->cld, cd.data(), sizeof(CLevel<double>) * nl, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(h->clf, cf.data(), sizeof(CLevel<float>) * nl, cudaMemcpyHostToDevice);
    if (e != cudaSuccess || !h->clsd) return e;
    // stacked batches: one instance's levels lstk.., instance by instance
    const int ls = nl - h->lstk;
    std::vector<CLevel<double>> sd((size_t)h->nsl * ls);
    std::vector<CLevel<float>> sf((size_t)h->nsl * ls);
    for (int y = 0; y < h->nsl; ++y)
        for (int l = h->lstk; l < nl; ++l) {
            const Level& L = h->lev[l];
            const Geom& gi = L.gi;
            auto inst = [&](auto C) {   // instance y's coefficient pointers
                const size_t f = (size_t)y * gi.nvel, c = (size_t)y * gi.ncell, e0 = (size_t)y * gi.esize[0];
                C.alpha += f;
                C.beta += f;
                C.invd_u += f;
                if (C.diag_u) C.diag_u += f;
                C.mu2_c += c;
                C.invd_p += c;
                C.mu_e[0] += e0;
                return C;
            };
            CLevel<double>& a = sd[(size_t)y * ls + (l - h->lstk)];
            CLevel<float>& b = sf[(size_t)y * ls + (l - h->lstk)];
            a = CLevel<double>{gi, inst(L.cdi), nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
            b = CLevel<float>{gi, inst(L.cfi), nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
            const size_t nu2 = (size_t)gi.nvel * gi.nvel, np2 = (size_t)gi.ncell * gi.ncell;
            if (L.smat_udi) {
                a.smat_u = L.smat_udi + y * nu2;
                b.smat_u = L.smat_ufi + y * nu2;
            }
            if (L.smat_pdi) {
                a.smat_p = L.smat_pdi + y * np2;
                b.smat_p = L.smat_pfi + y * np2;
            }
            a.smat_nc = b.smat_nc = (L.smat_udi || L.smat_pdi) ? SMAT_SWEEPS : 0;
        }
    e = cudaMemcpy(h->clsd, sd.data(), sizeof(CLevel<double>) * sd.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(h->clsf, sf.data(), sizeof(CLevel<float>) * sf.size(), cudaMemcpyHostToDevice);
}

// all coefficients from rho, mu (and gamma) on the finest level down
void build_coefficients(stk_handle* h, const double* rho, const double* mu, cudaStream_t s) {
    const Geom& g0 = h->lev[0].g;
    launch_fine_coefficients(g0, rho, mu, h->theta, h->lev[0].cd, s);
    if (h->bulk) launch_bulk_lambda(g0.ncell, h->gamma, mu, h->lev[0].cd.lam_c, s);
    for (size_t l = 1; l < h->lev.size(); ++l)
        launch_coarsen_coefficients(h->lev[l - 1].g, h->lev[l - 1].cd, h->lev[l].g, h->lev[l].cd, s);
    for (auto& L : h->lev) {
        launch_inverse_diagonals(L.g, L.cd, s);
        launch_convert_coefficients(L.g, L.cd, L.cf, s);
    }
    // stacked batches: the coarse levels' face coefficients instance by
    // instance, and each instance's coarse-solve matrices
    for (int l = h->lstk; h->clsd && l < (int)h->lev.size(); ++l) {
        Level& L = h->lev[l];
        launch_faces_by_instance<double>(L.gi, h->nsl, L.cd.alpha, L.cdi.alpha, s);
        launch_faces_by_instance<double>(L.gi, h->nsl, L.cd.beta, L.cdi.beta, s);
        launch_faces_by_instance<double>(L.gi, h->nsl, L.cd.invd_u, L.cdi.invd_u, s);
        launch_faces_by_instance<double>(L.gi, h->nsl, L.cd.diag_u, L.cdi.diag_u, s);
        launch_faces_by_instance<float>(L.gi, h->nsl, L.cf.alpha, L.cfi.alpha, s);
        launch_faces_by_instance<float>(L.gi, h->nsl, L.cf.beta, L.cfi.beta, s);
        launch_faces_by_instance<float>(L.gi, h->nsl, L.cf.invd_u, L.cfi.invd_u, s);
        if (L.smat_udi || L.smat_pdi) {
            const Geom& gi = L.gi;
            const size_t nu2 = (size_t)gi.nvel * gi.nvel, np2 = (size_t)gi.ncell * gi.ncell;
            for (int y = 0; y < h->nsl; ++y) {
                Coef<double> cd = L.cdi;
                Coef<float> cf = L.cfi;
                const size_t f = (size_t)y * gi.nvel, c = (size_t)y * gi.ncell, e0 = (size_t)y * gi.esize[0];
                cd.alpha += f; cd.beta += f; cd.invd_u += f; cd.diag_u += f;
                cd.mu2_c += c; cd.invd_p += c; cd.mu_e[0] += e0;
                cf.alpha += f; cf.beta += f; cf.invd_u += f;
                cf.mu2_c += c; cf.invd_p += c; cf.mu_e[0] += e0;
                if (L.smat_udi) {
                    launch_coarsest_matrix_vel<double>(gi, cd, SMAT_SWEEPS, L.smat_udi + y * nu2, s);
                    launch_coarsest_matrix_vel<float>(gi, cf, SMAT_SWEEPS, L.smat_ufi + y * nu2, s);
                }
                if (L.smat_pdi) {
                    launch_coarsest_matrix_cell<double>(gi, cd, SMAT_SWEEPS, L.smat_pdi + y * np2, s);
                    launch_coarsest_matrix_cell<float>(gi, cf, SMAT_SWEEPS, L.smat_pfi + y * np2, s);
                }
            }
        }
    }
    Level& Lc = h->lev.back();   // the coarse-solve matrices of both hierarchies
    if (Lc.smat_ud) {
        launch_coarsest_matrix_vel<double>(Lc.g, Lc.cd, SMAT_SWEEPS, Lc.smat_ud, s);
        launch_coarsest_matrix_vel<float>(Lc.g, Lc.cf, SMAT_SWEEPS, Lc.smat_uf, s);
    }
    if (Lc.smat_pd) {
        launch_coarsest_matrix_cell<double>(Lc.g, Lc.cd, SMAT_SWEEPS, Lc.smat_pd, s);
        launch_coarsest_matrix_cell<float>(Lc.g, Lc.cf, SMAT_SWEEPS, Lc.smat_pf, s);
    }
}

int create_handle(int dim, const int* n, double hh, const int* bc, int nsl, stk_handle** out);

}  // namespace

// ===================================================================== C ABI
extern "C" {

void stk_default_params(stk_solver_params* p) {
    if (!p) return;
    p->precond = STK_P1;
    p->restart = 10;
    p->rtol = 1e-10;
    p->maxit = 1000;
    p->precision = STK_FP64;
    p->nu = 2;
    p->ncoarse = 8;
    p->vcycles_u = 1;
    p->vcycles_p = 1;
}

const char* stk_last_error(const stk_handle* h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

long long stk_face_length(const stk_handle* h, int a) {
    if (!h || a < 0 || a >= h->dim) return -1;
    return h->lev[0].g.fsize[a];
}

long long stk_cell_length(const stk_handle* h) { return h ? h->lev[0].g.ncell : -1; }

int stk_create(int dim, const int* n, double hh, const int* bc, stk_handle** out) {
    return create_handle(dim, n, hh, bc, 1, out);
}

int stk_create_stacked(int dim, const int* n, double hh, const int* bc, int count, stk_handle** out) {
    if (out) *out = nullptr;
    if (dim != 2) return fail(nullptr, STK_ERR_ARG, "stacked batches are 2D");
    if (count < 1 || count > STK_MAX_STACK)
        return fail(nullptr, STK_ERR_ARG, "count must be 1..%d", STK_MAX_STACK);
    return create_handle(dim, n, hh, bc, count, out);
}

}  // extern "C"

namespace {

int create_handle(int dim, const int* n, double hh, const int* bc, int nsl, stk_handle** out) {
    stk_handle* h = nullptr;
    if (!out) return fail(nullptr, STK_ERR_ARG, "out is null");
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(nullptr, STK_ERR_ARG, "dim must be 2 or 3");
    if (!n || !bc) return fail(nullptr, STK_ERR_ARG, "null n or bc");
    if (!(hh > 0.0) || !std::isfinite(hh)) return fail(nullptr, STK_ERR_ARG, "h must be > 0");
    int nn[3] = {1, 1, 1}, bb[6] = {0, 0, 0, 0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        nn[a] = n[a];
        if (!is_pow2(n[a])) return fail(nullptr, STK_ERR_SIZE, "n[%d] = %d is not a power of two >= 2", a, n[a]);
        bb[2 * a] = bc[2 * a];
        bb[2 * a + 1] = bc[2 * a + 1];
        for (int sd = 0; sd < 2; ++sd)
            if (bb[2 * a + sd] < 0 || bb[2 * a + sd] > 2)
                return fail(nullptr, STK_ERR_ARG, "bad boundary code %d", bb[2 * a + sd]);
        if ((bb[2 * a] == STK_PERIODIC) != (bb[2 * a + 1] == STK_PERIODIC))
            return fail(nullptr, STK_ERR_ARG, "axis %d: periodic must be set on both sides", a);
    }
    long long total = nsl;
    for (int a = 0; a < dim; ++a) total *= nn[a];
    if (total * (dim + 1) > (1LL << 30)) return fail(nullptr, STK_ERR_SIZE, "grid too large");
    h = new stk_handle();
    cudaGetDevice(&h->device);
    h->dim = dim;
    h->nsl = nsl;
    int cur[3] = {nn[0], nn[1], nn[2]};
    double hl = hh;
    while (true) {
        Level L{};
        L.g = make_geom(dim, cur, hl, bb, nsl);
        h->lev.push_back(L);
        int mn = cur[0];
        for (int a = 1; a < dim; ++a) mn = cur[a] < mn ? cur[a] : mn;
        if (mn <= 2) break;
        for (int a = 0; a < dim; ++a) cur[a] /= 2;
        hl *= 2.0;
    }
#define CKC(call)                                                                   \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            fail(nullptr, STK_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
            stk_destroy(h);                                                         \
            return STK_ERR_CUDA;                                                    \
        }                                                                           \
    } while (0)
    for (auto& L : h->lev) {
        const Geom& g = L.g;
        CKC(dalloc(h, &L.cd.alpha, g.nvel));
        CKC(dalloc(h, &L.cd.beta, g.nvel));
        CKC(dalloc(h, &L.cd.mu2_c, g.ncell));
        CKC(dalloc(h, &L.cd.invd_u, g.nvel));
        CKC(dalloc(h, &L.cd.invd_p, g.ncell));
        CKC(dalloc(h, &L.cd.diag_u, g.nvel));
        L.cf.diag_u = nullptr;
        CKC(dalloc(h, &L.cf.alpha, g.nvel));
        CKC(dalloc(h, &L.cf.beta, g.nvel));
        CKC(dalloc(h, &L.cf.mu2_c, g.ncell));
        CKC(dalloc(h, &L.cf.invd_u, g.nvel));
        CKC(dalloc(h, &L.cf.invd_p, g.ncell));
        for (int p = 0; p < 3; ++p) {
            L.cd.mu_e[p] = nullptr;
            L.cf.mu_e[p] = nullptr;
            if (g.esize[p] > 0) {
                CKC(dalloc(h, &L.cd.mu_e[p], g.esize[p]));
                CKC(dalloc(h, &L.cf.mu_e[p], g.esize[p]));
            }
        }
        CKC(dalloc(h, &L.wd.phi_u, g.nvel));
        CKC(dalloc(h, &L.wd.rhs_u, g.nvel));
        CKC(dalloc(h, &L.wd.res_u, g.nvel));
        CKC(dalloc(h, &L.wd.phi_p, g.ncell));
        CKC(dalloc(h, &L.wd.rhs_p, g.ncell));
        CKC(dalloc(h, &L.wd.res_p, g.ncell));
        CKC(dalloc(h, &L.wd.alt_u, g.nvel));
        CKC(dalloc(h, &L.wd.alt_p, g.ncell));
        CKC(dalloc(h, &L.wf.phi_u, g.nvel));
        CKC(dalloc(h, &L.wf.rhs_u, g.nvel));
        CKC(dalloc(h, &L.wf.res_u, g.nvel));
        CKC(dalloc(h, &L.wf.phi_p, g.ncell));
        CKC(dalloc(h, &L.wf.rhs_p, g.ncell));
        CKC(dalloc(h, &L.wf.res_p, g.ncell));
        CKC(dalloc(h, &L.wf.alt_u, g.nvel));
        CKC(dalloc(h, &L.wf.alt_p, g.ncell));
    }
    if (nsl == 1) {   // (a stacked batch sweeps on its coarsest level)
        Level& Lc = h->lev.back();
        const size_t nu = (size_t)Lc.g.nvel, np = (size_t)Lc.g.ncell;
        if (nu <= (size_t)SMAT_MAX) {
            CKC(dalloc(h, &Lc.smat_ud, nu * nu));
            CKC(dalloc(h, &Lc.smat_uf, nu * nu));
        }
        if (np <= (size_t)SMAT_MAX) {
            CKC(dalloc(h, &Lc.smat_pd, np * np));
            CKC(dalloc(h, &Lc.smat_pf, np * np));
        }
    }
    // stacked batches: instance copies of the levels that the coarse-level
    // kernel may take (at most 65536 cells per instance, as stk_autotune)
    h->lstk = (int)h->lev.size();
    if (nsl > 1) {
        while (h->lstk > 0 && h->lev[h->lstk - 1].g.ncell / nsl <= 65536) --h->lstk;
        for (int l = h->lstk; l < (int)h->lev.size(); ++l) {
            Level& L = h->lev[l];
            const Geom& g = L.g;
            const int nn1[3] = {g.n[0], g.n[1], 1};
            const int bb1[6] = {g.bclo[0], g.bchi[0], g.bclo[1], g.bchi[1], 0, 0};
            L.gi = make_geom(dim, nn1, g.h, bb1, 1);
            const size_t nf = (size_t)L.gi.nvel * nsl;
            L.cdi = L.cd;
            L.cfi = L.cf;
            CKC(dalloc(h, &L.cdi.alpha, nf));
            CKC(dalloc(h, &L.cdi.beta, nf));
            CKC(dalloc(h, &L.cdi.invd_u, nf));
            CKC(dalloc(h, &L.cdi.diag_u, nf));
            CKC(dalloc(h, &L.cfi.alpha, nf));
            CKC(dalloc(h, &L.cfi.beta, nf));
            CKC(dalloc(h, &L.cfi.invd_u, nf));
            if (l + 1 == (int)h->lev.size()) {
                const size_t nu = (size_t)L.gi.nvel, np = (size_t)L.gi.ncell;
                if (nu <= (size_t)SMAT_MAX) {
                    CKC(dalloc(h, &L.smat_udi, nu * nu * nsl));
                    CKC(dalloc(h, &L.smat_ufi, nu * nu * nsl));
                }
                if (np <= (size_t)SMAT_MAX) {
                    CKC(dalloc(h, &L.smat_pdi, np * np * nsl));
                    CKC(dalloc(h, &L.smat_pfi, np * np * nsl));
                }
            }
        }
        if (h->lstk < (int)h->lev.size()) {
            const size_t nd = (size_t)nsl * (h->lev.size() - h->lstk);
            CKC(dalloc(h, &h->clsd, nd));
            CKC(dalloc(h, &h->clsf, nd));
        }
    }
    const Geom& g0 = h->lev[0].g;
    const int ns = g0.nvel + g0.ncell;
    h->smap.len[0] = g0.fsize[0] / nsl;
    h->smap.len[1] = g0.fsize[1] / nsl;
    h->smap.len[2] = g0.ncell / nsl;
    h->smap.off[0] = 0;
    h->smap.off[1] = g0.foff[1];
    h->smap.off[2] = g0.nvel;
    h->smap.nl = h->smap.len[0] + h->smap.len[1] + h->smap.len[2];
    CKC(dalloc(h, &h->pd.in, ns));
    CKC(dalloc(h, &h->pd.bc, g0.ncell));
    CKC(dalloc(h, &h->pd.tmpu, g0.nvel));
    CKC(dalloc(h, &h->pd.xs, g0.nvel));
    CKC(dalloc(h, &h->pd.ru, g0.nvel));
    CKC(dalloc(h, &h->pd.du, g0.nvel));
    CKC(dalloc(h, &h->pd.rp, g0.ncell));
    CKC(dalloc(h, &h->pd.dp, g0.ncell));
    CKC(dalloc(h, &h->pf.in, ns));
    CKC(dalloc(h, &h->pf.bc, g0.ncell));
    CKC(dalloc(h, &h->pf.tmpu, g0.nvel));
    CKC(dalloc(h, &h->pf.xs, g0.nvel));
    CKC(dalloc(h, &h->pf.ru, g0.nvel));
    CKC(dalloc(h, &h->pf.du, g0.nvel));
    CKC(dalloc(h, &h->pf.rp, g0.ncell));
    CKC(dalloc(h, &h->pf.dp, g0.ncell));
    CKC(dalloc(h, &h->bk, ns));
    CKC(dalloc(h, &h->xk, ns));
    CKC(dalloc(h, &h->tmp, ns));
    CKC(dalloc(h, &h->red, (size_t)RED_SCRATCH * nsl));
    CKC(dalloc(h, &h->rcnt, (size_t)nsl));
    for (int a = 0; a < g0.dim; ++a) CKC(dalloc(h, &h->sw.tc[a], g0.ncell));
    for (int p = 0; p < 3; ++p)
        if (g0.esize[p] > 0) CKC(dalloc(h, &h->sw.te[p], g0.esize[p]));
    CKC(dalloc(h, &h->rho0, g0.ncell));
    CKC(dalloc(h, &h->mu0, g0.ncell));
    CKC(dalloc(h, &h->dsc, (size_t)NDSC * nsl));
    {
        void* p = nullptr;
        CKC(cudaMallocHost(&p, sizeof(double) * 256));
        h->hpin = static_cast<double*>(p);
        static_assert(sizeof(GmState) % 8 == 0, "GmState records are packed as doubles");
        double* q = nullptr;
        CKC(dalloc(h, &q, sizeof(GmState) / 8 * nsl));
        h->gst = reinterpret_cast<GmState*>(q);
        CKC(dalloc(h, &h->gcond, GM_NCOND));
        CKC(dalloc(h, &h->gbar, 4));
        const long long budget = 2000000000LL;   // about one second at 2 GHz
        CKC(cudaMemcpy(h->gbar + 2, &budget, sizeof budget, cudaMemcpyHostToDevice));
        CKC(cudaMallocHost(&p, sizeof(GmState) * nsl));
        h->gst_host = static_cast<GmState*>(p);
        std::memset(h->gst_host, 0, sizeof(GmState) * nsl);
        CKC(cudaMallocHost(&p, sizeof(unsigned) * GM_NCOND));
        h->gcond_host = static_cast<unsigned*>(p);
        std::memset(h->gcond_host, 0, sizeof(unsigned) * GM_NCOND);
    }
    CKC(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    CKC(cudaStreamCreateWithFlags(&h->run, cudaStreamNonBlocking));
    CKC(cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&h->cyc, cudaEventDisableTiming));
    {   // level descriptors of the single-block coarse-level kernel
        const int nl = (int)h->lev.size();
        h->lcoarse_d = h->lcoarse_f = nl;
        h->lgrid_d = h->lgrid_f = nl;
        h->lcluster_d = h->lcluster_f = nl;
        // two-colour sweeps by default only in FP32 2D, where their halo
        // recomputation is small (measured; the autotuner decides per grid)
        h->lpair_d = nl;
        h->lpair_f = h->dim == 2 ? 0 : nl;
        // (a stacked batch: the cells of one instance, each has its own block)
        while (h->lcoarse_f > 0 && h->lev[h->lcoarse_f - 1].g.ncell / nsl <= COARSE_MAX_CELLS_F32) --h->lcoarse_f;
        while (h->lcoarse_d > 0 && h->lev[h->lcoarse_d - 1].g.ncell / nsl <= COARSE_MAX_CELLS_F64) --h->lcoarse_d;
        std::vector<CLevel<double>> cd(nl);
        std::vector<CLevel<float>> cf(nl);
        CKC(dalloc(h, &h->cld, nl));
        CKC(dalloc(h, &h->clf, nl));
        CKC(upload_clevels(h));
        prepare_coarse_kernels();
        CKC(cudaGetLastError());
    }
#undef CKC
    *out = h;
    return STK_OK;
}

}  // namespace

extern "C" {

int stk_destroy(stk_handle* h) {
    if (!h) return STK_OK;
    cudaDeviceSynchronize();
    clear_graphs(h);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->run) cudaStreamDestroy(h->run);
    if (h->join) cudaEventDestroy(h->join);
    if (h->cyc) cudaEventDestroy(h->cyc);
    for (void* p : h->allocs) cudaFree(p);
    if (h->hpin) cudaFreeHost(h->hpin);
    if (h->gst_host) cudaFreeHost(h->gst_host);
    if (h->gcond_host) cudaFreeHost(h->gcond_host);
    for (auto e : h->evpool) cudaEventDestroy(e);
    delete h;
    return STK_OK;
}

int stk_set_coefficients(stk_handle* h, const double* rho, const double* mu, double dt,
                         void* stream) {
    if (!h) return STK_ERR_ARG;
    Nvtx range("stk_set_coefficients");
    if (!rho || !mu) return fail(h, STK_ERR_ARG, "null rho or mu");
    if (!(dt > 0.0)) return fail(h, STK_ERR_ARG, "dt must be > 0 (+INFINITY for steady flow)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->device));
    const long long k0 = tl_launches;
    const Geom& g0 = h->lev[0].g;
    launch_check_fields(g0.ncell, rho, mu, h->red, h->dsc + DS_N2, s);
    CKL();
    CK(cudaMemcpyAsync(h->hpin, h->dsc + DS_N2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h->hpin[0] != 0.0) return fail(h, STK_ERR_NONFINITE, "rho or mu has %g non-finite entries", h->hpin[0]);
    if (h->hpin[1] != 0.0) return fail(h, STK_ERR_ARG, "rho <= 0 or mu < 0 at %g cells", h->hpin[1]);
    bool all_periodic = true;
    for (int a = 0; a < h->dim; ++a) all_periodic = all_periodic && g0.per[a];
    const double theta = std::isinf(dt) ? 0.0 : 1.0 / dt;
    if (theta == 0.0 && all_periodic)
        return fail(h, STK_ERR_ARG, "steady flow on an all-periodic grid (constant-velocity null space) is not supported");
    // The preconditioner graphs hold pointers only (coefficients and theta
    // are read from device memory), except that they contain the Poisson
    // solve or not: rebuild them only when theta changes between zero and
    // non-zero.
    if (!h->coef_set || (theta != 0.0) != (h->theta != 0.0)) clear_graphs(h);
    h->theta = theta;
    h->hpin[HP_THETA] = theta;
    CK(cudaMemcpyAsync(h->dsc + DS_THETA, h->hpin + HP_THETA, sizeof(double), cudaMemcpyHostToDevice, s));
    // rho and mu are kept so that stk_set_bulk_viscosity can rebuild
    CK(cudaMemcpyAsync(h->rho0, rho, sizeof(double) * g0.ncell, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(h->mu0, mu, sizeof(double) * g0.ncell, cudaMemcpyDeviceToDevice, s));
    build_coefficients(h, rho, mu, s);
    CKL();
    h->nkern += tl_launches - k0;
    CK(cudaStreamSynchronize(s));
    h->coef_set = true;
    return STK_OK;
}

int stk_set_bulk_viscosity(stk_handle* h, const double* gamma, void* stream) {
    if (!h) return STK_ERR_ARG;
    if (h->nsl > 1) return fail(h, STK_ERR_ARG, "not available on a stacked batch");
    if (!h->coef_set) return fail(h, STK_ERR_STATE, "coefficients not set");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->device));
    const long long k0 = tl_launches;
    const Geom& g0 = h->lev[0].g;
    const bool on = gamma != nullptr;
    if (on) {   // gamma finite and >= 0 (checked beside the stored rho > 0)
        launch_check_fields(g0.ncell, h->rho0, gamma, h->red, h->dsc + DS_N2, s);
        CKL();
        CK(cudaMemcpyAsync(h->hpin, h->dsc + DS_N2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (h->hpin[0] != 0.0) return fail(h, STK_ERR_NONFINITE, "gamma has %g non-finite entries", h->hpin[0]);
        if (h->hpin[1] != 0.0) return fail(h, STK_ERR_ARG, "gamma < 0 at %g cells", h->hpin[1]);
        if (!h->gamma) {   // first use: level-0 gamma and the lam hierarchy
            CK(dalloc(h, &h->gamma, g0.ncell));
            for (auto& L : h->lev) {
                CK(dalloc(h, &L.lam_d, L.g.ncell));
                CK(dalloc(h, &L.lam_f, L.g.ncell));
            }
        }
        CK(cudaMemcpyAsync(h->gamma, gamma, sizeof(double) * g0.ncell, cudaMemcpyDeviceToDevice, s));
    }
    if (on != h->bulk) {
        // the coefficient structs carry the lam pointers only while the bulk
        // term is on; graphs and level descriptors embed those structs
        clear_graphs(h);
        for (auto& L : h->lev) {
            L.cd.lam_c = on ? L.lam_d : nullptr;
            L.cf.lam_c = on ? L.lam_f : nullptr;
        }
        h->bulk = on;
        CK(upload_clevels(h));
    }
    build_coefficients(h, h->rho0, h->mu0, s);
    CKL();
    h->nkern += tl_launches - k0;
    CK(cudaStreamSynchronize(s));
    return STK_OK;
}

int stk_apply_operator(stk_handle* h, const double* const* x_u, const double* x_p,
                       double* const* y_u, double* y_p, void* stream) {
    if (!h) return STK_ERR_ARG;
    if (!h->coef_set) return fail(h, STK_ERR_STATE, "coefficients not set");
    int rc;
    if ((rc = check_ptrs(h, (const void* const*)x_u, x_p))) return rc;
    if ((rc = check_ptrs(h, (const void* const*)y_u, y_p))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->device));
    if ((rc = gather(h, x_u, x_p, h->xk, s))) return rc;
    {
        Scope sc(h, PF_MATVEC, bytes_matvec(h->lev[0].g, 8), s, stress_kernels(h->lev[0].g));
        launch_stokes_matvec_stress(h->lev[0].g, h->lev[0].cd, h->sw, h->xk, nullptr, h->tmp, s);
    }
    CKL();
    return scatter(h, h->tmp, y_u, y_p, s);
}

int stk_apply_preconditioner(stk_handle* h, int which, const double* const* b_u,
                             const double* b_p, double* const* x_u, double* x_p, void* stream) {
    if (!h) return STK_ERR_ARG;
    if (!h->coef_set) return fail(h, STK_ERR_STATE, "coefficients not set");
    if (which < STK_P1 || which > STK_P5) return fail(h, STK_ERR_ARG, "preconditioner must be 1..5");
    int rc;
    if ((rc = check_ptrs(h, (const void* const*)b_u, b_p))) return rc;
    if ((rc = check_ptrs(h, (const void* const*)x_u, x_p))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->device));
    if ((rc = gather(h, b_u, b_p, h->bk, s))) return rc;
    MGParams mp;
    apply_precond<double>(h, which, h->bk, h->tmp, mp, s);
    CKL();
    return scatter(h, h->tmp, x_u, x_p, s);
}

int stk_apply_preconditioner_params(stk_handle* h, const stk_solver_params* params,
                                    const double* const* b_u, const double* b_p,
                                    double* const* x_u, double* x_p, void* stream) {
    if (!h) return STK_ERR_ARG;
    if (!params) return fail(h, STK_ERR_ARG, "null params");
    if (!h->coef_set) return fail(h, STK_ERR_STATE, "coefficients not set");
    int rc;
    if ((rc = validate_params(h, *params))) return rc;
    if ((rc = check_ptrs(h, (const void* const*)b_u, b_p))) return rc;
    if ((rc = check_ptrs(h, (const void* const*)x_u, x_p))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->device));
    MGParams mp;
    mp.nu = params->nu;
    mp.ncoarse = params->ncoarse;
    mp.cu = params->vcycles_u;
    mp.cp = params->vcycles_p;
    if ((rc = gather(h, b_u, b_p, h->bk, s))) return rc;
    if (params->precision == STK_MIXED) {
        if ((rc = ensure_krylov(h, 1))) return rc;
        const int n = nstokes(h);
        launch_convert<double, float>(n, h->bk, h->pf.in, s);
        apply_precond<float>(h, params->precond, h->pf.in, h->Z[0], mp, s);
        launch_convert<float, double>(n, h->Z[0], h->tmp, s);
    } else {
        apply_precond<double>(h, params->precond, h->bk, h->tmp, mp, s);
    }
    CKL();
    return scatter(h, h->tmp, x_u, x_p, s);
}

int stk_subtract_boundary_terms(stk_handle* h, const double* const* u_wall,
                                const double* const* u_tan, double* const* b_u, double* b_p,
                                void* stream) {
    if (!h) return STK_ERR_ARG;
    if (h->nsl > 1) return fail(h, STK_ERR_ARG, "not available on a stacked batch");
    if (!h->coef_set) return fail(h, STK_ERR_STATE, "coefficients not set");
    int rc;
    if ((rc = check_ptrs(h, (const void* const*)b_u, b_p))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->device));
    const Level& L = h->lev[0];
    const Geom& g = L.g;
    const int n = nstokes(h);
    // M applied to the vector that holds only the normal wall velocities
    launch_zero<double>(n, h->xk, s);
    if (u_wall)
        for (int a = 0; a < g.dim; ++a)
            if (!g.per[a] && u_wall[a]) launch_copy_walls(g, a, u_wall[a], h->xk, s);
    launch_stokes_matvec_stress(g, L.cd, h->sw, h->xk, nullptr, h->tmp, s);
    h->nkern += stress_kernels(g);
    // tangential velocities of no-slip walls
    if (u_tan)
        for (int d = 0; d < g.dim; ++d) {
            if (g.per[d]) continue;
            for (int side = 0; side < 2; ++side) {
                if ((side ? g.bchi[d] : g.bclo[d]) != STK_NOSLIP) continue;
                for (int a = 0; a < g.dim; ++a) {
                    const double* U = u_tan[3 * (2 * d + side) + a];
                    if (a == d || !U) continue;
                    launch_wall_tangential(g, L.cd.mu_e[a + d - 1], d, side, a, U, h->tmp, s);
                }
            }
        }
    for (int a = 0; a < g.dim; ++a) launch_axpy<double>(g.fsize[a], -1.0, h->tmp + g.foff[a], b_u[a], s);
    launch_axpy<double>(g.ncell, -1.0, h->tmp + g.nvel, b_p, s);
    CKL();
    return STK_OK;
}

int stk_backward_euler_rhs(stk_handle* h, const double* const* u_n, const double* const* f,
                           double* const* b_u, void* stream) {
    if (!h) return STK_ERR_ARG;
    if (!h->coef_set) return fail(h, STK_ERR_STATE, "coefficients not set");
    if (!u_n || !b_u) return fail(h, STK_ERR_ARG, "null pointer");
    if (h->theta == 0.0) return fail(h, STK_ERR_STATE, "steady coefficients (dt = inf): no time step");
    const Geom& g = h->lev[0].g;
    for (int a = 0; a < g.dim; ++a)
        if (!u_n[a] || !b_u[a] || (f && !f[a])) return fail(h, STK_ERR_ARG, "null face array %d", a);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->device));
    for (int a = 0; a < g.dim; ++a)
        launch_inertial_rhs(g, a, h->lev[0].cd.alpha, u_n[a], f ? f[a] : nullptr, b_u[a], s);
    CKL();
    return STK_OK;
}

int stk_velocity_vcycle(stk_handle* h, const double* const* r_u, double* const* x_u,
                        void* stream) {
    if (!h) return STK_ERR_ARG;
    if (!h->coef_set) return fail(h, STK_ERR_STATE, "coefficients not set");
    if (!r_u || !x_u) return fail(h, STK_ERR_ARG, "null pointer");
    for (int a = 0; a < h->dim; ++a)
        if (!r_u[a] || !x_u[a]) return fail(h, STK_ERR_ARG, "null face array");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->device));
    const Geom& g = h->lev[0].g;
    for (int a = 0; a < g.dim; ++a)
        CK(cudaMemcpyAsync(h->bk + g.foff[a], r_u[a], sizeof(double) * g.fsize[a], cudaMemcpyDeviceToDevice, s));
    MGParams mp;
    vcycle_vel<double>(h, 0, h->bk, h->tmp, mp, s);
    CKL();
    for (int a = 0; a < g.dim; ++a)
        CK(cudaMemcpyAsync(x_u[a], h->tmp + g.foff[a], sizeof(double) * g.fsize[a], cudaMemcpyDeviceToDevice, s));
    return STK_OK;
}

int stk_pressure_vcycle(stk_handle* h, const double* r_p, double* x_p, void* stream) {
    if (!h) return STK_ERR_ARG;
    if (!h->coef_set) return fail(h, STK_ERR_STATE, "coefficients not set");
    if (!r_p || !x_p) return fail(h, STK_ERR_ARG, "null pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->device));
    MGParams mp;
    vcycle_cell<double>(h, 0, r_p, x_p, mp, s);
    CKL();
    return STK_OK;
}

int stk_solve(stk_handle* h, const stk_solver_params* params, const double* const* b_u,
              const double* b_p, double* const* x_u, double* x_p, stk_solve_info* info_out,
              void* stream) {
    stk_batch_io io{b_u, b_p, x_u, x_p};
    stk_handle* hs[1] = {h};
    if (!h) return STK_ERR_ARG;
    return stk_solve_batched(1, hs, params, &io, info_out, stream);
}

int stk_solve_batched(int count, stk_handle* const* hs, const stk_solver_params* params,
                      const stk_batch_io* io, stk_solve_info* infos, void* stream) {
    if (count < 1 || !hs || !io) return STK_ERR_ARG;
    Nvtx range(count == 1 ? "stk_solve" : "stk_solve_batched");
    stk_solver_params prm;
    stk_default_params(&prm);
    if (params) prm = *params;
    cudaStream_t us = static_cast<cudaStream_t>(stream);
    for (int i = 0; i < count; ++i) {
        stk_handle* h = hs[i];
        if (!h) return STK_ERR_ARG;
        if (!h->coef_set) return fail(h, STK_ERR_STATE, "coefficients not set");
        int rc;
        if ((rc = validate_params(h, prm))) return rc;
        if ((rc = check_ptrs(h, (const void* const*)io[i].b_u, io[i].b_p))) return rc;
        if ((rc = check_ptrs(h, (const void* const*)io[i].x_u, io[i].x_p))) return rc;
        for (int j = 0; j < i; ++j)
            if (hs[j] == h) return fail(h, STK_ERR_ARG, "a handle appears twice in one batch");
    }
    stk_handle* h0 = hs[0];
    int dev = h0->device;
    {
        stk_handle* h = h0;
        CK(cudaSetDevice(dev));
    }
    // one solve: the caller's stream; several: each handle's own stream,
    // forked from and joined back into the caller's stream
    std::vector<Inst> insts(count);
    cudaEvent_t e0, e1;
    {
        stk_handle* h = h0;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, us));
    }
    // one solve: the caller's stream, each GMRES cycle one graph launch.
    // Several: each instance on its handle's own stream.  Up to
    // BATCH_CYCLE_GRAPHS instances (e.g. one stacked handle per grid size)
    // each run their cycles as graph launches independently of the others;
    // larger batches gate the cycles' phases by the host for the whole batch
    // at once (measured faster for 64 single-instance handles than 64
    // independent cycle graphs)
    const bool fork = count > 1;
    for (int i = 0; i < count; ++i) {
        Inst& it = insts[i];
        it.h = hs[i];
        it.s = fork ? hs[i]->run : us;
        if (fork) cudaStreamWaitEvent(it.s, e0, 0);
        int rc = gather(it.h, io[i].b_u, io[i].b_p, it.h->bk, it.s);
        if (!rc) rc = gather(it.h, io[i].x_u, io[i].x_p, it.h->xk, it.s);
        if (rc) finish(&it, rc);
    }
    gmres_lockstep(insts, prm, count <= BATCH_CYCLE_GRAPHS);
    int worst = STK_OK;
    for (int i = 0; i < count; ++i) {
        Inst& it = insts[i];
        // a stacked batch hands back every instance's iterate (stk_stack_info
        // says which converged), also when one of them failed
        const bool partial = it.h->nsl > 1 && (it.rc == STK_ERR_NONFINITE || it.rc == STK_ERR_TIMEOUT);
        if (it.rc == STK_OK || it.rc == STK_ERR_NOT_CONVERGED || partial) {
            int rc2 = scatter(it.h, it.h->xk, io[i].x_u, io[i].x_p, it.s);
            if (rc2) it.rc = rc2;
        }
        if (fork) {
            cudaEventRecord(it.h->join, it.s);
            cudaStreamWaitEvent(us, it.h->join, 0);
        }
        if (it.rc == STK_ERR_NOT_CONVERGED)
            fail(it.h, it.rc, "not converged after %d iterations (residual %.3e)", it.info.iterations,
                 it.info.true_residual);
        if (it.rc != STK_OK && (worst == STK_OK || worst == STK_ERR_NOT_CONVERGED)) worst = it.rc;
    }
    cudaEventRecord(e1, us);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int i = 0; i < count; ++i) {
        insts[i].info.solve_ms = ms;
        insts[i].info.status = insts[i].rc;
        stk_handle* h = insts[i].h;
        for (int y = 0; y < (int)h->sinfo.size(); ++y) {
            stk_solve_info& f = h->sinfo[y];
            f.solve_ms = ms;
            switch (h->gst_host[y].state) {
            case GM_CONVERGED: f.status = STK_OK; break;
            case GM_MAXIT: f.status = STK_ERR_NOT_CONVERGED; break;
            case GM_NONFINITE: f.status = STK_ERR_NONFINITE; break;
            case GM_TIMEOUT: f.status = STK_ERR_TIMEOUT; break;
            default: f.status = insts[i].rc == STK_OK ? STK_ERR_STATE : insts[i].rc;
            }
        }
        if (infos) infos[i] = insts[i].info;
    }
    return worst;
}

int stk_get_schedule(const stk_handle* h, int precision, stk_schedule* out) {
    if (!h || !out || (precision != STK_FP64 && precision != STK_MIXED)) return STK_ERR_ARG;
    out->coarse_level = precision == STK_FP64 ? h->lcoarse_d : h->lcoarse_f;
    out->threads = precision == STK_FP64 ? h->tpb_d : h->tpb_f;
    out->pair_level = precision == STK_FP64 ? h->lpair_d : h->lpair_f;
    out->grid_level = precision == STK_FP64 ? h->lgrid_d : h->lgrid_f;
    out->cluster_level = precision == STK_FP64 ? h->lcluster_d : h->lcluster_f;
    return STK_OK;
}

int stk_set_schedule(stk_handle* h, int precision, const stk_schedule* sc) {
    if (!h) return STK_ERR_ARG;
    if (!sc || (precision != STK_FP64 && precision != STK_MIXED))
        return fail(h, STK_ERR_ARG, "bad schedule arguments");
    if (sc->coarse_level < 0 || sc->coarse_level > (int)h->lev.size())
        return fail(h, STK_ERR_ARG, "coarse_level must be in 0..%d", (int)h->lev.size());
    if (sc->threads != 64 && sc->threads != 128 && sc->threads != 256 && sc->threads != 512)
        return fail(h, STK_ERR_ARG, "threads must be 64, 128, 256 or 512");
    if (sc->pair_level < 0 || sc->pair_level > (int)h->lev.size())
        return fail(h, STK_ERR_ARG, "pair_level must be in 0..%d", (int)h->lev.size());
    if (sc->grid_level < 0 || sc->grid_level > (int)h->lev.size())
        return fail(h, STK_ERR_ARG, "grid_level must be in 0..%d", (int)h->lev.size());
    if (h->nsl > 1 && sc->grid_level < sc->coarse_level)
        return fail(h, STK_ERR_ARG, "a stacked batch has no persistent multi-block V-cycle (grid_level >= coarse_level)");
    if (sc->cluster_level < 0 || sc->cluster_level > (int)h->lev.size())
        return fail(h, STK_ERR_ARG, "cluster_level must be in 0..%d", (int)h->lev.size());
    if (h->nsl > 1 && sc->cluster_level < sc->coarse_level)
        return fail(h, STK_ERR_ARG, "a stacked batch has no cluster V-cycle (cluster_level >= coarse_level)");
    clear_graphs(h);
    if (precision == STK_FP64) {
        h->lcoarse_d = sc->coarse_level;
        h->tpb_d = sc->threads;
        h->lpair_d = sc->pair_level;
        h->lgrid_d = sc->grid_level;
        h->lcluster_d = sc->cluster_level;
    } else {
        h->lcoarse_f = sc->coarse_level;
        h->tpb_f = sc->threads;
        h->lpair_f = sc->pair_level;
        h->lgrid_f = sc->grid_level;
        h->lcluster_f = sc->cluster_level;
    }
    return STK_OK;
}

}  // extern "C"

namespace {
// time `reps` replays of the velocity + pressure V-cycle pair in precision T
// captured as one graph, with the current schedule
template <typename T>
int time_vcycles(stk_handle* h, int reps, cudaStream_t s, float* ms) {
    PBuf<T>& B = pbuf_of<T>(h);
    const Level& L = h->lev[0];
    MGParams mp;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    vcycle_vel<T>(h, 0, B.in, B.xs, mp, h->cap);
    vcycle_cell<T>(h, 0, B.in + L.g.nvel, B.bc, mp, h->cap);
    h->capturing = false;
    CK(cudaStreamEndCapture(h->cap, &g));
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, STK_ERR_CUDA, "autotune instantiate: %s", cudaGetErrorString(e));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaGraphLaunch(ex, s);   // warm-up
    // the fastest of three batches of reps launches: a schedule is judged by
    // what it can do, not by a transient slowdown during one batch
    *ms = 1e30f;
    for (int batch = 0; batch < 3; ++batch) {
        cudaEventRecord(a, s);
        for (int r = 0; r < reps; ++r) cudaGraphLaunch(ex, s);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float t = 0.f;
        cudaEventElapsedTime(&t, a, b);
        *ms = t < *ms ? t : *ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaGraphExecDestroy(ex);
    CKL();
    return STK_OK;
}
}  // namespace

extern "C" {

int stk_autotune(stk_handle* h, int precision, stk_schedule* best, void* stream) {
    if (!h) return STK_ERR_ARG;
    Nvtx range("stk_autotune");
    if (!h->coef_set) return fail(h, STK_ERR_STATE, "coefficients not set");
    if (precision != STK_FP64 && precision != STK_MIXED) return fail(h, STK_ERR_ARG, "bad precision");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->device));
    const bool prof = h->prof;
    h->prof = false;
    stk_schedule cur;
    stk_get_schedule(h, precision, &cur);
    stk_schedule bs = cur;
    float bms = 1e30f;
    const int nl = (int)h->lev.size();
    const int threads[3] = {128, 256, 512};
    for (int lc = 0; lc <= nl; ++lc) {
        // the single-block kernel only pays on small levels
        if (lc < nl && h->lev[lc].g.ncell / h->nsl > 65536) continue;
        // two-colour kernels from level 0, 1 or 2, or not at all (pair_level
        // = lc); the colour block size only matters below pair_level
        int pls[4], npl = 0;
        for (int p = 0; p < 3 && p < lc; ++p) pls[npl++] = p;
        pls[npl++] = lc;
        // the cluster kernel (cluster_level) from one or two levels above
        // the single-block one, or not (= lc).  The persistent multi-block
        // kernel (grid_level) is not tried: it was slower than the cluster
        // kernel on every grid measured (it stays available to
        // stk_set_schedule).
        int gls[5], cls[5], ngl = 0;
        gls[ngl] = lc;
        cls[ngl++] = lc;
        for (int d = 1; d <= 2 && lc - d >= 0 && h->nsl == 1; ++d)
            if (h->lev[lc - d].g.ncell <= 262144) {
                gls[ngl] = lc;
                cls[ngl++] = lc - d;
            }
        for (int k = 0; k < npl; ++k)
            for (int gi = 0; gi < ngl; ++gi)
            for (int ti = 0; ti < (pls[k] == 0 ? 1 : 3); ++ti) {
                const int top = std::min(gls[gi], cls[gi]);   // first level run as one launch
                if (top < lc && pls[k] > top && pls[k] < lc) continue;
                stk_schedule c{lc, threads[ti], pls[k], gls[gi], cls[gi]};
                int rc = stk_set_schedule(h, precision, &c);
                if (rc) { h->prof = prof; return rc; }
                float ms = 0.f;
                rc = precision == STK_FP64 ? time_vcycles<double>(h, 3, s, &ms)
                                           : time_vcycles<float>(h, 3, s, &ms);
                if (rc) {   // a schedule that cannot be captured or launched is skipped
                    cudaGetLastError();
                    continue;
                }
                if (ms < bms) {
                    bms = ms;
                    bs = c;
                }
            }
    }
    h->prof = prof;
    int rc = stk_set_schedule(h, precision, &bs);
    if (best) *best = bs;
    return rc;
}

int stk_profile(stk_handle* h, int enable) {
    if (!h) return STK_ERR_ARG;
    prof_flush(h);
    if (enable) {
        for (int k = 0; k < STK_NPROF; ++k) {
            h->plaunch[k] = 0;
            h->pms[k] = 0.0;
            h->pbytes[k] = 0.0;
            h->pflops[k] = 0.0;
        }
    }
    h->prof = enable != 0;
    return STK_OK;
}

long long stk_kernel_launches(const stk_handle* h) { return h ? h->nkern : -1; }

int stk_gradient(stk_handle* h, const double* const* u, const double* const* lambda,
                 double* dL_dlogmu, double* dL_drho, void* stream) {
    if (!h) return STK_ERR_ARG;
    if (h->nsl > 1) return fail(h, STK_ERR_ARG, "not available on a stacked batch");
    if (!h->coef_set) return fail(h, STK_ERR_STATE, "coefficients not set");
    if (h->bulk) return fail(h, STK_ERR_STATE, "the gradient is defined for the stress form without bulk viscosity");
    if (!u || !lambda || !dL_dlogmu || !dL_drho) return fail(h, STK_ERR_ARG, "null pointer");
    for (int a = 0; a < h->dim; ++a)
        if (!u[a] || !lambda[a]) return fail(h, STK_ERR_ARG, "null face array");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->device));
    const Geom& g = h->lev[0].g;
    for (int a = 0; a < g.dim; ++a) {
        CK(cudaMemcpyAsync(h->bk + g.foff[a], u[a], sizeof(double) * g.fsize[a], cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(h->tmp + g.foff[a], lambda[a], sizeof(double) * g.fsize[a], cudaMemcpyDeviceToDevice, s));
    }
    {
        Scope sc(h, PF_ALG, 8.0 * (2.0 * g.nvel + 3.0 * g.ncell), s);
        launch_gradient(g, h->mu0, h->theta, h->bk, h->tmp, dL_dlogmu, dL_drho, s);
    }
    CKL();
    return STK_OK;
}

long long stk_bounds_violations(long long* first_kind, long long* first_index, int reset) {
#ifdef STK_BOUNDS_CHECK
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    long long (*readers[])(long long*, int) = {oob_kernels, oob_pair, oob_stress, oob_coarse};
    long long total = 0;
    bool have = false;
    for (auto rd : readers) {
        long long first[2] = {0, 0};
        const long long c = rd(first, reset);
        if (c < 0) return -1;
        if (c > 0 && !have) {
            have = true;
            if (first_kind) *first_kind = first[0];
            if (first_index) *first_index = first[1];
        }
        total += c;
    }
    return total;
#else
    (void)first_kind;
    (void)first_index;
    (void)reset;
    return -1;
#endif
}

int stk_bounds_selftest(void* stream) {
#ifdef STK_BOUNDS_CHECK
    launch_oob_selftest(7, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? STK_OK : STK_ERR_CUDA;
#else
    (void)stream;
    return STK_ERR_STATE;
#endif
}

int stk_set_graphs(stk_handle* h, int enable) {
    if (!h) return STK_ERR_ARG;
    clear_graphs(h);
    h->use_graphs = enable != 0;
    return STK_OK;
}

int stk_widen(const float* x, double* y, long long n, void* stream) {
    if (!x || !y || n < 0 || n > 0x7fffffffLL) return STK_ERR_ARG;
    if (n == 0) return STK_OK;
    launch_convert<float, double>((int)n, x, y, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? STK_OK : STK_ERR_CUDA;
}

int stk_graphs_in_use(const stk_handle* h) { return h ? (h->use_graphs ? 1 : 0) : STK_ERR_ARG; }

int stk_set_wait_budget(stk_handle* h, long long cycles) {
    if (!h) return STK_ERR_ARG;
    if (cycles < 0) return fail(h, STK_ERR_ARG, "the wait budget must be >= 0");
    CK(cudaSetDevice(h->device));
    CK(cudaMemcpy(h->gbar + 2, &cycles, sizeof cycles, cudaMemcpyHostToDevice));
    return STK_OK;
}

int stk_wait_status(stk_handle* h, int reset) {
    if (!h) return STK_ERR_ARG;
    CK(cudaSetDevice(h->device));
    CK(cudaDeviceSynchronize());
    int v = 0;
    CK(cudaMemcpy(&v, &h->gst->wait_status, sizeof v, cudaMemcpyDeviceToHost));
    if (reset) CK(cudaMemset(&h->gst->wait_status, 0, sizeof v));
    return v == 0 ? STK_OK : STK_ERR_TIMEOUT;
}

int stk_solve_history(const stk_handle* h, int kind, double* out, int cap) {
    return stk_stack_history(h, 0, kind, out, cap);
}

int stk_stack_history(const stk_handle* h, int instance, int kind, double* out, int cap) {
    if (!h || (kind != 0 && kind != 1) || cap < 0 || instance < 0 || instance >= h->nsl) return STK_ERR_ARG;
    const auto& all = kind == 0 ? h->hist_true : h->hist_est;
    if (instance >= (int)all.size()) return 0;
    const std::vector<double>& v = all[instance];
    if (out)
        for (int i = 0; i < cap && i < (int)v.size(); ++i) out[i] = v[i];
    return (int)v.size();
}

int stk_stack_info(const stk_handle* h, int instance, stk_solve_info* info) {
    if (!h || !info || instance < 0 || instance >= h->nsl) return STK_ERR_ARG;
    if (instance >= (int)h->sinfo.size()) return STK_ERR_STATE;
    *info = h->sinfo[instance];
    return STK_OK;
}

int stk_stack_count(const stk_handle* h) { return h ? h->nsl : STK_ERR_ARG; }

int stk_remove_mean(stk_handle* h, const double* x_p, double* y_p, void* stream) {
    if (!h) return STK_ERR_ARG;
    if (!x_p || !y_p) return fail(h, STK_ERR_ARG, "null pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(h->device));
    const int nc = h->lev[0].g.ncell;
    {
        Scope sc(h, PF_MEAN, 2.0 * sizeof(double) * nc, s, 2);
        cell_sum<double>(h, nc, x_p, h->dsc + DS_SUM + 6, s);
        sub_mean<double>(h, nc, x_p, y_p, h->dsc + DS_SUM + 6, s);
    }
    CKL();
    return STK_OK;
}

int stk_profile_read(stk_handle* h, int k, const char** name, long long* launches, double* ms,
                     double* bytes, double* flops) {
    if (!h || k < 0 || k >= STK_NPROF) return -1;
    prof_flush(h);
    if (name) *name = kProfNames[k];
    if (launches) *launches = h->plaunch[k];
    if (ms) *ms = h->pms[k];
    if (bytes) *bytes = h->pbytes[k];
    if (flops) *flops = h->pflops[k];
    return STK_OK;
}

}  // extern "C"
