// Device-resident control of restarted GMRES (Sec. 3.2) and of its flexible
// variant (Sec. 4): the Hessenberg least-squares problem, its Givens
// rotations, the residual estimate, the stopping decisions and the
// back-substitution live in a GmState record in device memory (one per
// instance of a stacked batch), updated by one-block kernels, a thread per
// record, between the vector kernels of each Arnoldi step.
//
// Every decision is written to st->cond[], its OR over the instances to a
// group word and, inside a CUDA graph, to the conditional node that gates the
// next phase (cudaGraphSetConditional), so one GMRES cycle of m Arnoldi
// steps runs as one graph launch with no host round trip; the host reads
// the records once per cycle.  Without a graph (profiling, host-gated
// batches) the host reads the group words after each phase instead.  The
// arithmetic is the textbook one (Saad): column j of the Hessenberg matrix is
// rotated by the j earlier rotations, a new rotation zeroes h_{j+1,j}, the
// right-hand side g = beta e_1 is rotated alongside, |g_{j+1}| is the
// residual estimate, and y solves the k x k triangular system R y = g.
#include "internal.cuh"

#include <cmath>

namespace stk {
namespace {

// Each kernel runs as one block; thread y < nsl updates the record of
// instance y (a stacked batch has one record per instance, a single solve
// one).  A decision v_y is written to st[y].cond[slot]; its OR over the
// instances goes to gc[slot] and, inside a graph, to the conditional node
// that gates the next phase: a phase runs while any instance needs it, and
// the kernels of the phase leave the others alone.  Every thread reaches
// every set_cond (a block-wide OR).
__device__ __forceinline__ void set_cond(GmState* st, bool mine, unsigned* gc, int slot, unsigned v,
                                         cudaGraphConditionalHandle hc, int use) {
    if (mine) st->cond[slot] = v;
    const unsigned any = __syncthreads_or(mine && v != 0u) ? 1u : 0u;
    if (threadIdx.x == 0) {
        gc[slot] = any;
        if (use) cudaGraphSetConditional(hc, any);
    }
}

__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

// a bounded device wait (a grid barrier of the persistent V-cycle) ran out:
// the iteration stops
__device__ __forceinline__ bool timed_out(GmState* st) {
    if (st->wait_status == 0) return false;
    if (st->state == GM_RUNNING) st->state = GM_TIMEOUT;
    return true;
}

__device__ __forceinline__ void fail_nonfinite(GmState* st, int why) {
    if (st->state == GM_RUNNING) {
        st->state = GM_NONFINITE;
        st->why = why;
    }
}

// solve start: ||b|| from its square; a zero right-hand side is solved by x = 0
__global__ void k_gm_begin(GmState* st0, int nsl, unsigned* gc, const double* __restrict__ bn2,
                           int dstride, double rtol, int maxit, int m, int flex) {
    pdl_entry();
    const int y = threadIdx.x;
    if (y == 0)
        for (int i = 0; i < GM_NCOND; ++i) gc[i] = 0;
    if (y >= nsl) return;
    GmState* st = st0 + y;
    st->bnorm = sqrt(bn2[(size_t)y * dstride]);
    st->rtol = rtol;
    st->maxit = maxit;
    st->m = m;
    st->flex = flex;
    st->iterations = 0;
    st->restarts = 0;
    st->k = 0;
    st->nhist = 0;
    st->nest = 0;
    st->why = 0;
    st->rnorm = st->beta = st->target = st->est = 0.0;
    st->wait_status = 0;
    if (!finite(st->bnorm)) {
        st->state = GM_NONFINITE;
        st->why = GM_WHY_RHS;
    } else {
        st->state = st->bnorm == 0.0 ? GM_CONVERGED : GM_RUNNING;
    }
    for (int i = 0; i < GM_NCOND; ++i) st->cond[i] = 0;
}

// graph cycles: the stopping test runs only while an instance is running (a
// finished solve costs this one kernel per cycle)
__global__ void k_gm_gate(GmState* st0, int nsl, unsigned* gc, cudaGraphConditionalHandle hchk) {
    pdl_entry();
    const int y = threadIdx.x;
    const bool mine = y < nsl;
    GmState* st = st0 + (mine ? y : 0);
    set_cond(st, mine, gc, GM_COND_CHK, (mine && st->state == GM_RUNNING) ? 1u : 0u, hchk, 1);
}

// cycle start, after r = b - M x and ||r||^2: record the true residual, stop
// on convergence, maxit or a non-finite residual; otherwise open the cycle
__global__ void k_gm_check(GmState* st0, int nsl, unsigned* gc, const double* __restrict__ rn2,
                           int dstride, cudaGraphConditionalHandle hpre, int use) {
    pdl_entry();
    const int y = threadIdx.x;
    const bool mine = y < nsl;
    GmState* st = st0 + (mine ? y : 0);
    unsigned go = 0;
    if (mine) {
        st->k = 0;
        st->cond[GM_COND_CHK] = 1;
        st->cond[GM_COND_FIN] = 0;
        for (int j = 0; j < GM_MMAX; ++j) st->cond[GM_COND_STEP0 + j] = 0;
        timed_out(st);
        if (st->state == GM_RUNNING) {
            const double rn = sqrt(rn2[(size_t)y * dstride]);
            st->rnorm = rn;
            if (!finite(rn)) {
                fail_nonfinite(st, GM_WHY_RESIDUAL);
            } else {
                if (st->nhist < GM_NHIST) st->hist[st->nhist] = rn / st->bnorm;
                ++st->nhist;
                if (rn <= st->rtol * st->bnorm) st->state = GM_CONVERGED;
                else if (st->iterations >= st->maxit) st->state = GM_MAXIT;
                else go = 1;
            }
        }
    }
    if (y == 0) {
        gc[GM_COND_CHK] = 1;
        gc[GM_COND_FIN] = 0;
        for (int j = 0; j < GM_MMAX; ++j) gc[GM_COND_STEP0 + j] = 0;
    }
    set_cond(st, mine, gc, GM_COND_PRE, go, hpre, use);
}

// after the cycle's first basis vector r0 (left: P^{-1} r, flexible: r) and,
// for the left form, ||r0||^2: beta, the cycle's target and 1 / beta
__global__ void k_gm_start(GmState* st0, int nsl, unsigned* gc, const double* __restrict__ vn2,
                           int dstride, cudaGraphConditionalHandle h0, int use0,
                           cudaGraphConditionalHandle hfin, int usefin) {
    pdl_entry();
    const int y = threadIdx.x;
    const bool mine = y < nsl;
    GmState* st = st0 + (mine ? y : 0);
    unsigned go = 0;
    if (mine) {
        timed_out(st);
        if (st->state == GM_RUNNING) {
            const double beta = st->flex ? st->rnorm : sqrt(vn2[(size_t)y * dstride]);
            st->beta = beta;
            if (!finite(beta)) {
                fail_nonfinite(st, GM_WHY_PRECOND);
            } else if (beta == 0.0) {
                // the preconditioned residual vanished while the true one did not
                st->state = GM_MAXIT;
            } else {
                // flexible: the Arnoldi residual is the true residual; left: the
                // preconditioned residual must fall by the factor the true
                // residual still needs
                st->target = st->flex ? st->rtol * st->bnorm : beta * (st->rtol * st->bnorm / st->rnorm);
                st->g[0] = beta;
                for (int i = 1; i <= st->m; ++i) st->g[i] = 0.0;
                st->inv_scale = 1.0 / beta;
                ++st->restarts;
                go = 1;
            }
        }
    }
    set_cond(st, mine, gc, GM_COND_STEP0, go, h0, use0);
    set_cond(st, mine, gc, GM_COND_FIN, go, hfin, usefin);
}

// Arnoldi step j done: h[0..j] = projections, *n2 = ||w||^2 after them (of
// each instance at stride dstride).  Rotate the new column, form the next
// rotation, update g and the estimate, and decide whether step j + 1 runs.
// An instance whose step j is not open is left as it is.
__device__ unsigned gm_step_one(GmState* st, int j, const double* hcol, const double* n2) {
    if (!st->cond[GM_COND_STEP0 + j]) return 0u;
    if (timed_out(st)) st->k = 0;   // no update from a cycle whose preconditioner failed
    if (st->state != GM_RUNNING) return 0u;
    double* H = st->H + j * (GM_MMAX + 1);   // column j, rows 0..j+1
    bool ok = finite(*n2);
    for (int i = 0; i <= j; ++i) {
        H[i] = hcol[i];
        ok = ok && finite(H[i]);
    }
    const double hnext = sqrt(*n2);
    H[j + 1] = hnext;
    ++st->iterations;
    st->k = j + 1;
    if (!ok) {
        fail_nonfinite(st, GM_WHY_ARNOLDI);
        st->k = 0;
        return 0u;
    }
    for (int i = 0; i < j; ++i) {
        const double t = st->cs[i] * H[i] + st->sn[i] * H[i + 1];
        H[i + 1] = -st->sn[i] * H[i] + st->cs[i] * H[i + 1];
        H[i] = t;
    }
    const double a = H[j], b = H[j + 1];
    const double r = hypot(a, b);
    st->cs[j] = r == 0.0 ? 1.0 : a / r;
    st->sn[j] = r == 0.0 ? 0.0 : b / r;
    H[j] = st->cs[j] * a + st->sn[j] * b;
    H[j + 1] = 0.0;
    st->g[j + 1] = -st->sn[j] * st->g[j];
    st->g[j] = st->cs[j] * st->g[j];
    const double est = fabs(st->g[j + 1]);
    st->est = est;
    if (st->nest < GM_NEST) st->est_hist[st->nest] = est / st->bnorm;
    ++st->nest;
    st->inv_scale = hnext > 0.0 ? 1.0 / hnext : 1.0;
    const bool more = est > st->target && hnext > 0.0 && st->iterations < st->maxit;
    return more ? 1u : 0u;
}

__global__ void k_gm_step(GmState* st0, int nsl, unsigned* gc, int j, const double* __restrict__ hcol,
                          const double* __restrict__ n2, int dstride, cudaGraphConditionalHandle hn,
                          int use) {
    pdl_entry();
    const int y = threadIdx.x;
    const bool mine = y < nsl;
    GmState* st = st0 + (mine ? y : 0);
    unsigned more = 0;
    if (mine) more = gm_step_one(st, j, hcol + (size_t)y * dstride, n2 + (size_t)y * dstride);
    if (j + 1 < GM_MMAX && j + 1 < st0->m) set_cond(st, mine, gc, GM_COND_STEP0 + j + 1, more, hn, use);
}

// cycle end: y = R^{-1} g over the k steps taken (k = 0 after a failure or
// for an instance that did not run the cycle: no update)
__global__ void k_gm_finish(GmState* st0, int nsl) {
    pdl_entry();
    if ((int)threadIdx.x >= nsl) return;
    GmState* st = st0 + threadIdx.x;
    const int k = st->k;
    bool ok = true;
    for (int i = k - 1; i >= 0; --i) {
        double s = st->g[i];
        for (int c = i + 1; c < k; ++c) s -= st->H[c * (GM_MMAX + 1) + i] * st->y[c];
        st->y[i] = s / st->H[i * (GM_MMAX + 1) + i];
        ok = ok && finite(st->y[i]);
    }
    if (!ok) {
        fail_nonfinite(st, GM_WHY_UPDATE);
        st->k = 0;
    }
}

// x *= *s
__global__ void __launch_bounds__(256) k_scal_dev(int n, double* __restrict__ x,
                                                  const double* __restrict__ s) {
    pdl_entry();
    const double a = *s;
    for (int t = blockIdx.x * 256 + threadIdx.x; t < n; t += gridDim.x * 256) x[t] *= a;
}

// one block with a thread per instance (whole warps)
inline dim3 ctl_block(int nsl) { return dim3(32 * ((nsl + 31) / 32)); }

}  // namespace

void launch_gm_begin(GmState* st, int nsl, unsigned* gc, const double* bn2, int dstride, double rtol,
                     int maxit, int m, int flex, cudaStream_t s) {
    launch_pdl(k_gm_begin, dim3(1), ctl_block(nsl), s, st, nsl, gc, bn2, dstride, rtol, maxit, m, flex);
}
void launch_gm_check(GmState* st, int nsl, unsigned* gc, const double* rn2, int dstride,
                     cudaGraphConditionalHandle hpre, int use, cudaStream_t s) {
    launch_pdl(k_gm_check, dim3(1), ctl_block(nsl), s, st, nsl, gc, rn2, dstride, hpre, use);
}
void launch_gm_gate(GmState* st, int nsl, unsigned* gc, cudaGraphConditionalHandle hchk, cudaStream_t s) {
    launch_pdl(k_gm_gate, dim3(1), ctl_block(nsl), s, st, nsl, gc, hchk);
}
void launch_gm_start(GmState* st, int nsl, unsigned* gc, const double* vn2, int dstride,
                     cudaGraphConditionalHandle h0, int use0, cudaGraphConditionalHandle hfin, int usefin,
                     cudaStream_t s) {
    launch_pdl(k_gm_start, dim3(1), ctl_block(nsl), s, st, nsl, gc, vn2, dstride, h0, use0, hfin, usefin);
}
void launch_gm_step(GmState* st, int nsl, unsigned* gc, int j, const double* hcol, const double* n2,
                    int dstride, cudaGraphConditionalHandle hn, int use, cudaStream_t s) {
    launch_pdl(k_gm_step, dim3(1), ctl_block(nsl), s, st, nsl, gc, j, hcol, n2, dstride, hn, use);
}
void launch_gm_finish(GmState* st, int nsl, cudaStream_t s) {
    launch_pdl(k_gm_finish, dim3(1), ctl_block(nsl), s, st, nsl);
}
void launch_scale_dev(int n, double* x, const double* a, cudaStream_t s) {
    const int nb = (n + 256 * 8 - 1) / (256 * 8);   // about eight values per thread
    launch_pdl(k_scal_dev, dim3(nb < 1 ? 1 : (nb > KRY_BLOCKS ? KRY_BLOCKS : nb)), dim3(256), s, n, x, a);
}

}  // namespace stk
