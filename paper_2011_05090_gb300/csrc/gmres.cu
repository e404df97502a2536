// RGS-Arnoldi (Alg. 3), restarted randomized GMRES (Sec. 4.2, Eq. hls) and the FP64
// CGS2-GMRES comparator (projector (I - Q Q^T)^2, Sec. 1.2).
//
// The basis is stored as q'_i with q_i = q'_i sigma_i, sigma_i = 1 / r_ii.  The product
// w'_{i+1} = A q'_i and its sketch are formed before r_ii is known; w_{i+1} = sigma_i w'_{i+1}
// follows from the one-synchronisation "lag" of Sec. 2.4: the least-squares kernel scales the
// sketch p'_{i+1} by 1 / r_ii when it appends column i, and the update of column i + 1 scales
// its input.  (Unnormalised Krylov columns would grow like ||A||^i and overflow FP32 storage.)
// One Arnoldi step is three launches: the fused update + sketch of column i (Alg. 2 steps 3-4),
// the product with the sketch fused in (Alg. 3 step 3, Alg. 2 step 1), and the least-squares
// kernel (steps 2, 5, 6 plus the Givens rotation of H(:, i-1) = R(0:i+1, i), Sec. 4.1).
// A converged or broken-down cycle raises a stop word that turns the remaining launches of
// the cycle into no-ops; the host reads it once per cycle with the true residual.
#include "common.cuh"
#include "givens.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <new>
#include <vector>

using namespace rgsdev;

struct rgs_arnoldi_obj {
    rgs_handle h = nullptr;
    rgs_sketch_obj* sk = nullptr;
    int64_t n = 0;
    int mmax = 0;
    int qtype = 0;
    int fine64 = 0;          // RGS_FP64_FINE: FP64 transform sums, products and least squares for any qtype
    int ls64 = 0;            // RGS_FP64_LS: FP64 least squares (and Givens) for any qtype
    int64_t ldq = 0;
    int ncols = 0;           // columns appended so far (public step-by-step interface)
    DevBuf Q;                // n x mmax in qtype
    DevBuf lsbuf;
    LSState ls{};
    DevBuf R;                // mmax x mmax
    DevBuf gv;               // cs, sn, g, Hr, y, cy
    DevBuf wbuf;             // w' (FP64 or double-float pairs), n
    DevBuf spart, ppart;     // partial sketches of q'_i and of w'_{i+1}
    DevBuf vdf;              // A's values split into double-float pairs
    DevBuf work;             // r (n), norm partials, scalars
    DevBuf jac;              // Jacobi: diag(A)^{-1} (n) and the values of A D^{-1} (nnz)
    DevBuf Z;                // flexible preconditioning: z'_i = M(q'_i), n x mmax FP32 (a caller's
                             // M: FP64 for an FP64 basis; one column when it is not flexible)
    DevBuf pct;              // a caller's linear M, not flexible: Q y (FP64, n) at the end of a cycle
    const SellView* sell = nullptr;        // A in SELL-32 form for the fused product (rgmres_solve)
    unsigned long long* trace = nullptr;   // RGS_TRACE: least-squares timestamps of step i at
    size_t tstride = 0;                    // trace + i * tstride (the latest cycle's steps)
};

namespace {

template <class F>
rgs_status guarded(rgs_handle h, F&& f) {
    try {
        f();
        if (h) h->last_error.clear();
        return RGS_OK;
    } catch (const RgsError& e) {
        if (h) h->last_error = e.msg;
        return e.status;
    } catch (const std::bad_alloc&) {
        if (h) h->last_error = "host allocation failed";
        return RGS_ERR_ALLOC;
    } catch (...) {
        if (h) h->last_error = "unexpected exception";
        return RGS_ERR_INVALID_ARG;
    }
}

size_t dsize(int t) { return t == RGS_F64 ? 8 : (t == RGS_F32 ? 4 : 2); }

void check_csr(const rgs_csr* A, int64_t n) {
    RGS_REQUIRE(A != nullptr && A->rowptr && A->colind && A->val, "null CSR array");
    RGS_REQUIRE(A->n == n && A->nnz >= 0, "CSR size differs from the sketch's n");
}

// Allocate everything an Arnoldi object needs for a basis of mmax columns.
void arnoldi_alloc(rgs_arnoldi_obj* a) {
    rgs_context* h = a->h;
    const int k = a->sk->k, m = a->mmax;
    a->ldq = (a->n + 7) & ~(int64_t)7;
    a->Q.ensure(dsize(a->qtype) * (size_t)a->ldq * m);
    rgs_ls_alloc(a->lsbuf, k, m, h->num_sms, h->num_sms * kUpdMaxBlocksPerSm,
                 a->qtype != RGS_F64 && !a->fine64 && !a->ls64, &a->ls);
    a->R.ensure(sizeof(double) * (size_t)m * m);
    a->gv.ensure(sizeof(double) * (4 * (size_t)m + 2 + (size_t)m * m + 2 * (size_t)m));
    double* g = a->gv.as<double>();
    a->ls.cs = g;
    a->ls.sn = g + m;
    a->ls.g = g + 2 * m;
    a->ls.Hr = g + 3 * m + 2;
    a->ls.R = a->R.as<double>();
    a->ls.ldr = m;
    a->ls.ctl = h->ctl.as<int>();
    a->wbuf.ensure(sizeof(double) * (size_t)a->n);
    const size_t parts = (size_t)h->num_sms * kUpdMaxBlocksPerSm * k * sizeof(double);
    a->spart.ensure(parts);
    a->ppart.ensure(parts);
    a->work.ensure(sizeof(double) * ((size_t)a->n + 8 * (size_t)h->num_sms + 16 + (size_t)k));
}

double* y_buf(rgs_arnoldi_obj* a) { return a->ls.Hr + (size_t)a->mmax * a->mmax; }
double* cy_buf(rgs_arnoldi_obj* a) { return y_buf(a) + a->mmax; }

void reset_cycle(rgs_arnoldi_obj* a) {
    rgs_context* h = a->h;
    RGS_CUDA(cudaMemsetAsync(h->ctl.as<int>() + kStopWord, 0, 2 * sizeof(int), h->stream));
    rgs_ls_reset(h, a->ls);
    RGS_CUDA(cudaMemsetAsync(a->R.ptr, 0, a->R.bytes, h->stream));
    RGS_CUDA(cudaMemsetAsync(a->gv.ptr, 0, a->gv.bytes, h->stream));
}

// Double-float transform sums and products: SRHT sketches of FP32 / BF16 bases unless FP64 is asked for.
bool sketch_is_df(const rgs_arnoldi_obj* a) {
    return a->sk->kind == RGS_SKETCH_SRHT && a->qtype != RGS_F64 && !a->fine64;
}

double s_scale(const rgs_sketch_obj* sk) { return sk->kind == RGS_SKETCH_SRHT ? 1.0 / std::sqrt((double)sk->k) : 1.0; }

// Steps 3-4 for column i from the input column w (FP64 or double-float) scaled by *wscale, into spart.
int launch_update(rgs_arnoldi_obj* a, int i, const void* w, int w_df, const double* wscale = nullptr,
                  bool no_gauss = false) {
    UpdateLaunch L{};
    L.n = a->n;
    L.ncols = i;
    L.Q = a->Q.ptr;
    L.ldq = a->ldq;
    L.qtype = a->qtype;
    L.w = reinterpret_cast<const double*>(w);
    L.ldw = a->n;
    L.wcols = 1;
    L.w_df = w_df;
    L.wscale = wscale;
    L.coef = a->ls.coef;
    L.qout = a->Q.as<char>() + dsize(a->qtype) * (size_t)i * a->ldq;
    L.df_sketch = sketch_is_df(a) ? 1 : 0;
    L.no_gauss = no_gauss ? 1 : 0;
    int np = 0;
    rgs_launch_update_sketch(a->h, a->sk, L, a->spart.as<double>(), &np, a->h->ctl.as<int>());
    return np;
}

// w' = A v (+ sketch of w' into ppart) for v = q'_col (or the vector v of type vtype when
// given); returns the number of partial sketches.
int launch_product(rgs_arnoldi_obj* a, const rgs_csr& A, int col, const void* v = nullptr, int vtype = -1,
                   bool sketch = true) {
    rgs_context* h = a->h;
    const void* x = v ? v : a->Q.as<char>() + dsize(a->qtype) * (size_t)col * a->ldq;
    const int xtype = v ? vtype : a->qtype;
    if (a->sk->kind == RGS_SKETCH_SRHT) {
        const int dfm = sketch_is_df(a) ? 1 : 0;
        return rgs_launch_spmv(h, A, a->vdf.ptr, x, xtype, a->wbuf.ptr, dfm, a->sk, a->ppart.as<double>(),
                               h->ctl.as<int>(), nullptr, a->sell);
    }
    rgs_launch_spmv(h, A, nullptr, x, xtype, a->wbuf.ptr, 0, nullptr, nullptr, h->ctl.as<int>());
    if (!sketch) return 0;
    UpdateLaunch L{};
    L.n = a->n;
    L.qtype = RGS_F64;
    L.w = a->wbuf.as<double>();
    L.ldw = a->n;
    L.wcols = 1;
    int np = 0;
    rgs_launch_update_sketch(h, a->sk, L, a->ppart.as<double>(), &np, h->ctl.as<int>());
    return np;
}

// The inner test ends a cycle once the Givens residual estimate falls below
// inner_factor * rtol * ||b|| (sketched norm for RGMRES).  With a reduced-precision basis the
// true residual of the updated x can stay above that estimate; a cycle that stopped on the
// test but left the true residual above rtol tightens the test of the following cycles by
// the ratio (target / true residual), so that restarts keep making progress.
void tighten_inner(double& stop_tol, int cycles, int last_steps, int m, double rel, const rgmres_opts& o) {
    if (cycles == 0 || stop_tol <= 0.0 || last_steps >= m || rel <= o.rtol || !(rel > 0.0)) return;
    stop_tol *= std::min(1.0, o.inner_factor * o.rtol / rel);
}

void launch_ls(rgs_arnoldi_obj* a, int i, int sparts, bool solve, int pparts, bool gmres, double stop_tol) {
    LSStep s{};
    s.i = i;
    s.append = 1;
    s.s_part = a->spart.as<double>();
    s.s_nparts = sparts;
    s.s_scale = s_scale(a->sk);
    s.s_df = sketch_is_df(a) ? 1 : 0;
    s.solve = solve ? 1 : 0;
    s.xcol = i + 1;
    s.p_part = a->ppart.as<double>();
    s.p_nparts = pparts;
    s.p_scale = s_scale(a->sk);
    s.p_df = sketch_is_df(a) ? 1 : 0;
    s.pnorm_idx = i + 1;
    s.p_lag = 1;                    // p_{i+1} = Theta (A q'_i) / r_ii
    s.givens = gmres ? 1 : 0;
    s.arnoldi = 1;
    s.stop_tol = stop_tol;
    s.trace = a->trace ? a->trace + a->tstride * (size_t)i : nullptr;
    rgs_launch_ls(a->h, a->ls, s);
}

struct Scalars {
    double* r;        // n
    double* part;     // norm partials (8 per SM)
    double* val;      // 16 device scalars: [0] ||r||, [1] ||b||, [2] ||Theta b||
    double* kvec;     // k entries: Theta b
};

Scalars scalars(rgs_arnoldi_obj* a) {
    double* w = a->work.as<double>();
    double* val = w + a->n + 8 * (size_t)a->h->num_sms;
    return {w, w + a->n, val, val + 16};
}

__global__ void scale_vec_kernel(int64_t n, double* w, const double* scale) {
    const double s = *scale;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] *= s;
}

}  // namespace

extern "C" {

rgs_status rgs_arnoldi_create(rgs_handle h, rgs_sketch s, int64_t n, int32_t mmax, rgs_dtype qtype,
                              int32_t flags, rgs_arnoldi* out) {
    if (!h || !s || !out) return RGS_ERR_INVALID_ARG;
    *out = nullptr;
    rgs_arnoldi_obj* a = new (std::nothrow) rgs_arnoldi_obj();
    if (!a) return RGS_ERR_ALLOC;
    rgs_status st = guarded(h, [&] {
        RGS_REQUIRE(qtype == RGS_F64 || qtype == RGS_F32 || qtype == RGS_BF16, "unknown qtype");
        RGS_REQUIRE(n == s->n, "n differs from the sketch's n");
        RGS_REQUIRE(mmax >= 1 && mmax <= s->k && mmax <= 1024 && mmax <= n, "need 1 <= mmax <= min(k, n, 1024)");
        RGS_REQUIRE((flags & ~(RGS_FP64_FINE | RGS_FP64_LS)) == 0, "unknown flags");
        a->h = h;
        a->sk = s;
        a->n = n;
        a->mmax = mmax;
        a->qtype = qtype;
        a->fine64 = (flags & RGS_FP64_FINE) ? 1 : 0;
        a->ls64 = (flags & RGS_FP64_LS) ? 1 : 0;
        arnoldi_alloc(a);
    });
    if (st != RGS_OK) {
        delete a;
        return st;
    }
    *out = a;
    return RGS_OK;
}

// Like rgs_sketch_destroy: releases device memory only and never touches the handle.
rgs_status rgs_arnoldi_destroy(rgs_arnoldi a) {
    if (!a) return RGS_ERR_INVALID_ARG;
    delete a;
    return RGS_OK;
}

// Alg. 3 steps 1-2: iteration 1 of Alg. 2 on w_1.
rgs_status rgs_arnoldi_start(rgs_handle h, rgs_arnoldi a, const double* w1) {
    if (!h || !a || !w1) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_CUDA(cudaMemsetAsync(h->ctl.ptr, 0, kCtlWords * sizeof(int), h->stream));
        reset_cycle(a);
        const int np = launch_update(a, 0, w1, 0);
        LSStep s{};
        s.i = 0;
        s.append = 1;
        s.s_part = a->spart.as<double>();
        s.s_nparts = np;
        s.s_scale = s_scale(a->sk);
        s.s_df = sketch_is_df(a) ? 1 : 0;
        rgs_launch_ls(h, a->ls, s);
        a->ncols = 1;
        int ctl[2];
        RGS_CUDA(cudaMemcpyAsync(ctl, h->ctl.ptr, sizeof(ctl), cudaMemcpyDeviceToHost, h->stream));
        RGS_CUDA(cudaStreamSynchronize(h->stream));
        if (ctl[0] != 0) throw RgsError{(rgs_status)ctl[0], "first Arnoldi column failed"};
    });
}

// Alg. 3 steps 3-4: w_i = A q_{i-1} (or the caller's w), then iteration i of Alg. 2.
rgs_status rgs_arnoldi_step(rgs_handle h, rgs_arnoldi a, const rgs_csr* A, const double* w) {
    if (!h || !a) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_REQUIRE(a->ncols >= 1, "rgs_arnoldi_start first");
        RGS_REQUIRE(a->ncols < a->mmax, "the basis is full (mmax columns)");
        RGS_REQUIRE(A != nullptr || w != nullptr, "need A or w");
        const int i = a->ncols;
        const double* wi = w;
        if (A) {
            // w_i = A q_{i-1} = sigma_{i-1} A q'_{i-1}: FP64 product, then scale
            check_csr(A, a->n);
            const void* x = a->Q.as<char>() + dsize(a->qtype) * (size_t)(i - 1) * a->ldq;
            rgs_launch_spmv(h, *A, nullptr, x, a->qtype, a->wbuf.ptr, 0, nullptr, nullptr, h->ctl.as<int>());
            const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((a->n + 255) / 256, 4 * h->num_sms));
            scale_vec_kernel<<<grid, 256, 0, h->stream>>>(a->n, a->wbuf.as<double>(), a->ls.sigma + (i - 1));
            RGS_CUDA(cudaGetLastError());
            wi = a->wbuf.as<double>();
        }
        // p_i = Theta w_i (FP64 sketch), then the pure least-squares solve with i reflectors
        UpdateLaunch L{};
        L.n = a->n;
        L.qtype = RGS_F64;
        L.w = wi;
        L.ldw = a->n;
        L.wcols = 1;
        int pp = 0;
        rgs_launch_update_sketch(h, a->sk, L, a->ppart.as<double>(), &pp, h->ctl.as<int>());
        LSStep s{};
        s.i = i;
        s.solve = 1;
        s.xcol = i;
        s.p_part = a->ppart.as<double>();
        s.p_nparts = pp;
        s.p_scale = s_scale(a->sk);
        s.pnorm_idx = i;
        rgs_launch_ls(h, a->ls, s);
        // Alg. 2 steps 3-4, then steps 5-6
        UpdateLaunch U{};
        U.n = a->n;
        U.ncols = i;
        U.Q = a->Q.ptr;
        U.ldq = a->ldq;
        U.qtype = a->qtype;
        U.w = wi;
        U.ldw = a->n;
        U.wcols = 1;
        U.coef = a->ls.coef;
        U.qout = a->Q.as<char>() + dsize(a->qtype) * (size_t)i * a->ldq;
        U.df_sketch = sketch_is_df(a) ? 1 : 0;
        int np = 0;
        rgs_launch_update_sketch(h, a->sk, U, a->spart.as<double>(), &np, h->ctl.as<int>());
        LSStep t{};
        t.i = i;
        t.append = 1;
        t.s_part = a->spart.as<double>();
        t.s_nparts = np;
        t.s_scale = s_scale(a->sk);
        t.s_df = sketch_is_df(a) ? 1 : 0;
        rgs_launch_ls(h, a->ls, t);
        int ctl[2];
        RGS_CUDA(cudaMemcpyAsync(ctl, h->ctl.ptr, sizeof(ctl), cudaMemcpyDeviceToHost, h->stream));
        RGS_CUDA(cudaStreamSynchronize(h->stream));
        if (ctl[0] != 0) {
            RGS_CUDA(cudaMemsetAsync(h->ctl.ptr, 0, 2 * sizeof(int), h->stream));
            throw RgsError{(rgs_status)ctl[0], "Arnoldi step " + std::to_string(i) + ": " +
                                                   rgs_status_string((rgs_status)ctl[0])};
        }
        a->ncols = i + 1;
    });
}

rgs_status rgs_arnoldi_get(rgs_handle h, rgs_arnoldi a, int32_t* ncols, double* R_host, int64_t ldr,
                           double* qscale_host) {
    if (!h || !a) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        if (ncols) *ncols = a->ncols;
        const int m = a->ncols;
        if (R_host && m > 0) {
            RGS_REQUIRE(ldr >= m, "ldr too small");
            RGS_CUDA(cudaMemcpy2DAsync(R_host, sizeof(double) * ldr, a->R.ptr, sizeof(double) * a->mmax,
                                       sizeof(double) * m, m, cudaMemcpyDeviceToHost, h->stream));
        }
        if (qscale_host && m > 0)
            RGS_CUDA(cudaMemcpyAsync(qscale_host, a->ls.sigma, sizeof(double) * m, cudaMemcpyDeviceToHost, h->stream));
        RGS_CUDA(cudaStreamSynchronize(h->stream));
    });
}

rgs_status rgs_arnoldi_basis(rgs_arnoldi a, void** Q, int64_t* ldq) {
    if (!a || !Q || !ldq) return RGS_ERR_INVALID_ARG;
    *Q = a->Q.ptr;
    *ldq = a->ldq;
    return RGS_OK;
}

rgs_status rgmres_solve(rgs_handle h, rgs_sketch s, const rgs_csr* A, const double* b, double* x,
                        const rgmres_opts* opts, rgmres_info* info) {
    if (!h || !s || !opts) return RGS_ERR_INVALID_ARG;
    if (info) {
        info->cycles = info->total_steps = info->converged = info->sell = info->sketch_refreshes = 0;
        info->status = RGS_OK;
        info->rel_residual = NAN;
    }
    bool converged = false;
    rgs_status st = guarded(h, [&] {
        check_csr(A, s->n);
        RGS_REQUIRE(b && x, "null b or x");
        RGS_REQUIRE(opts->restart >= 1 && opts->restart + 1 <= s->k && opts->restart < 1024,
                    "need 1 <= restart < min(k, 1024)");
        RGS_REQUIRE(opts->max_cycles >= 0 && opts->rtol >= 0.0, "bad max_cycles or rtol");
        RGS_REQUIRE((opts->flags & ~(RGS_FP64_FINE | RGS_FP64_LS)) == 0, "unknown flags");
        const int m = opts->restart;
        rgs_arnoldi_obj obj;
        obj.h = h;
        obj.sk = s;
        obj.n = s->n;
        obj.mmax = m + 1;
        obj.qtype = opts->qtype;
        obj.fine64 = (opts->flags & RGS_FP64_FINE) ? 1 : 0;
        obj.ls64 = (opts->flags & RGS_FP64_LS) ? 1 : 0;
        arnoldi_alloc(&obj);
        // Right preconditioning A M, x = x0 + M (Q y) (Sec. 5.3 preconditions A_f P_f from the right).
        // Jacobi, M = D^{-1}: the Arnoldi operator is A D^{-1} (column-scaled values), and the
        // solution update applies D^{-1}.  Learned network (nonlinear): flexible GMRES, z'_i = M(q'_i)
        // kept in Z, w' = A z'_i and x = x0 + Z y.  A caller's M: the same when flexible, else
        // one z per step and x = x0 + M (Q y).
        const int pk = h->precond_kind;
        RGS_REQUIRE(pk == RGS_PRECOND_NONE || pk == RGS_PRECOND_JACOBI || pk == RGS_PRECOND_LEARNED_CONV ||
                        pk == RGS_PRECOND_CALLBACK,
                    "unknown preconditioner");
        const bool learned = pk == RGS_PRECOND_LEARNED_CONV;
        const bool callback = pk == RGS_PRECOND_CALLBACK;
        const bool cb_flex = callback && h->precond_flexible != 0;
        const rgs_callback_precond cb = h->precond_cb;
        const int ztype = obj.qtype == RGS_F64 ? RGS_F64 : RGS_F32;
        auto apply_cb = [&](const void* v, int vtype, void* z) {
            const int32_t rc = cb.apply(cb.user, s->n, v, vtype, z, ztype, (void*)h->stream);
            if (rc != 0) throw RgsError{RGS_ERR_CALLBACK, "preconditioner callback returned " + std::to_string(rc)};
        };
        if (callback) {
            RGS_REQUIRE(cb.apply != nullptr, "preconditioner callback not set");
            obj.Z.ensure((size_t)dsize(ztype) * (size_t)obj.ldq * (cb_flex ? obj.mmax : 1));
            if (!cb_flex) obj.pct.ensure(sizeof(double) * (size_t)s->n);
        }
        rgs_csr Apc = *A;
        const double* dinv = nullptr;
        if (pk == RGS_PRECOND_JACOBI) {
            obj.jac.ensure(sizeof(double) * ((size_t)s->n + (size_t)std::max<int64_t>(A->nnz, 1)));
            double* jd = obj.jac.as<double>();
            rgs_launch_jacobi_setup(h, *A, jd, jd + s->n);
            dinv = jd;
            Apc.val = jd + s->n;
        }
        if (learned) {
            RGS_REQUIRE(h->precond_net != nullptr && h->precond_field != nullptr, "learned preconditioner not set");
            RGS_REQUIRE(rgs_convnet_grid_points(h->precond_net) == s->n,
                        "the network's H x W grid must have n points");
            obj.Z.ensure(sizeof(float) * (size_t)obj.ldq * obj.mmax);
        }
        DevBuf vdf_pc;                       // double-float values of A D^{-1}
        // The fused product with the SRHT reads A in SELL-32 form when its padding is small
        // (RGS_SELL=0 in the environment: CSR); A D^{-1} shares the structure, with its own values.
        SellBuf sell;
        SellView sview, sview_pc;
        const char* sell_env = std::getenv("RGS_SELL");
        const int dfm = sketch_is_df(&obj) ? 1 : 0;
        bool use_sell = false;
        if (s->kind == RGS_SKETCH_SRHT && !(sell_env && sell_env[0] == '0')) {
            try {                              // no room for the SELL-32 copy: the CSR product
                use_sell = rgs_build_sell(h, *A, dfm, sell);
            } catch (const RgsError& e) {
                if (e.status != RGS_ERR_ALLOC) throw;
                use_sell = false;
            }
        }
        if (use_sell) {
            sview.nslices = sell.nslices;
            sview.off = sell.off.as<int64_t>();
            sview.col = sell.col.as<int32_t>();
            sview.val = sell.val.ptr;
            sview_pc = sview;
            if (pk == RGS_PRECOND_JACOBI) {
                rgs_fill_sell_values(h, *A, Apc.val, dfm, sell, vdf_pc);
                sview_pc.val = vdf_pc.ptr;
            }
            obj.sell = &sview;
            if (info) info->sell = 1;
        } else if (dfm) {
            obj.vdf.ensure(8 * (size_t)std::max<int64_t>(A->nnz, 1));
            rgs_csr_split_df(h, A->val, A->nnz, obj.vdf.ptr);
            if (pk == RGS_PRECOND_JACOBI) {
                vdf_pc.ensure(8 * (size_t)std::max<int64_t>(A->nnz, 1));
                rgs_csr_split_df(h, Apc.val, A->nnz, vdf_pc.ptr);
            }
        }
        bool use_pc = pk != RGS_PRECOND_NONE;
        double prev_rel = INFINITY;
        int fallback_cycle = -1;
        // w' = A M q'_i (or A q'_i once the preconditioner is off), with its sketch
        auto product = [&](int i, bool sketch) -> int {
            if (use_pc && callback) {
                char* z = obj.Z.as<char>() + (cb_flex ? (size_t)dsize(ztype) * (size_t)i * obj.ldq : 0);
                apply_cb(obj.Q.as<char>() + dsize(obj.qtype) * (size_t)i * obj.ldq, obj.qtype, z);
                return launch_product(&obj, *A, i, z, ztype, sketch);
            }
            if (use_pc && learned) {
                float* z = obj.Z.as<float>() + (size_t)i * obj.ldq;
                rgs_convnet_apply_precond(h, h->precond_net, h->precond_field,
                                          obj.Q.as<char>() + dsize(obj.qtype) * (size_t)i * obj.ldq, obj.qtype, z);
                return launch_product(&obj, *A, i, z, RGS_F32, sketch);
            }
            if (use_pc) {
                void* keep = obj.vdf.ptr;
                if (vdf_pc.ptr && !obj.sell) obj.vdf.ptr = vdf_pc.ptr;
                if (obj.sell) obj.sell = &sview_pc;
                const int np = launch_product(&obj, Apc, i, nullptr, -1, sketch);
                obj.vdf.ptr = keep;
                if (obj.sell) obj.sell = &sview;
                return np;
            }
            return launch_product(&obj, *A, i, nullptr, -1, sketch);
        };
        // Gaussian sketch: Theta q'_i and Theta (A q'_i) in one pass over Theta (Sec. 2.4's single
        // synchronisation per step; the k x n matrix is read once per step instead of twice)
        const bool gauss2 = s->kind == RGS_SKETCH_GAUSSIAN;
        const bool trace = std::getenv("RGS_TRACE") != nullptr;
        PhaseTimer timer(h, trace);          // RGS_TRACE: device time of the update, product and LS launches
        auto step = [&](int i, const void* w, int w_df, const double* wscale, bool with_product, int& sp, int& pp) {
            if (trace && !(gauss2 && with_product)) {
                timer.start(0);
                sp = launch_update(&obj, i, w, w_df, wscale);
                timer.stop(0);
                if (with_product) {
                    timer.start(1);
                    pp = product(i, true);
                    timer.stop(1);
                }
                return;
            }
            if (gauss2 && with_product) {
                launch_update(&obj, i, w, w_df, wscale, true);
                product(i, false);
                const void* qi = obj.Q.as<char>() + dsize(obj.qtype) * (size_t)i * obj.ldq;
                sp = pp = rgs_launch_gauss_sketch2(h, obj.sk, s->n, qi, obj.qtype, obj.wbuf.as<double>(),
                                                   obj.spart.as<double>(), obj.ppart.as<double>(), h->ctl.as<int>());
            } else {
                sp = launch_update(&obj, i, w, w_df, wscale);
                if (with_product) pp = product(i, true);
            }
        };
        Scalars sc = scalars(&obj);
        if (trace) {
            obj.tstride = (size_t)rgs_ls_grid(h) * kLsTraceSlots;
            h->trace.ensure(sizeof(unsigned long long) * obj.tstride * (size_t)(m + 1));
            RGS_CUDA(cudaMemsetAsync(h->trace.ptr, 0, sizeof(unsigned long long) * obj.tstride * (size_t)(m + 1),
                                     h->stream));
            obj.trace = h->trace.as<unsigned long long>();
        }
        h->launches = 0;
        RGS_CUDA(cudaMemsetAsync(h->ctl.ptr, 0, kCtlWords * sizeof(int), h->stream));
        // ||b|| and ||Theta b|| (the inner stopping test compares the sketched residual with the latter)
        rgs_launch_norm(h, s->n, b, sc.part, sc.val + 1);
        {
            UpdateLaunch L{};
            L.n = s->n;
            L.qtype = RGS_F64;
            L.w = b;
            L.ldw = s->n;
            L.wcols = 1;
            int np = 0;
            rgs_launch_update_sketch(h, s, L, obj.ppart.as<double>(), &np, nullptr);
            rgs_launch_reduce_partials(h, obj.ppart.as<double>(), np, s->k, 1, s_scale(s), sc.kvec, s->k);
            rgs_launch_norm(h, s->k, sc.kvec, sc.part, sc.val + 2);
        }
        double hv[3];
        RGS_CUDA(cudaMemcpyAsync(hv, sc.val, sizeof(hv), cudaMemcpyDeviceToHost, h->stream));
        RGS_CUDA(cudaStreamSynchronize(h->stream));
        const double bnorm = hv[1], sbnorm = hv[2];
        RGS_REQUIRE(bnorm > 0.0 && std::isfinite(bnorm), "b must be nonzero and finite");
        double stop_tol = (opts->fixed_steps ? -1.0 : opts->inner_factor * opts->rtol * sbnorm);
        int cycles = 0, total = 0, refreshes = 0;
        double rel = NAN;
        struct SketchOwner {                 // a refreshed Theta, destroyed with the solve
            rgs_sketch p = nullptr;
            void reset(rgs_sketch q) {
                if (p) rgs_sketch_destroy(p);
                p = q;
            }
            ~SketchOwner() { reset(nullptr); }
        } fresh;
        for (;;) {
            rgs_launch_residual(h, *A, x, b, sc.r, sc.part, sc.val);     // true FP64 residual
            int ctlv[8];
            RGS_CUDA(cudaMemcpyAsync(hv, sc.val, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            RGS_CUDA(cudaMemcpyAsync(ctlv, h->ctl.ptr, sizeof(ctlv), cudaMemcpyDeviceToHost, h->stream));
            RGS_CUDA(cudaStreamSynchronize(h->stream));
            if (ctlv[0] != 0) throw RgsError{(rgs_status)ctlv[0], "device status in cycle " + std::to_string(cycles)};
            if (cycles > 0) total += ctlv[kStepsWord];
            rel = hv[0] / bnorm;
            tighten_inner(stop_tol, cycles, ctlv[kStepsWord], m, rel, *opts);
            if (info && info->history) info->history[cycles] = rel;
            if (!std::isfinite(rel)) throw RgsError{RGS_ERR_NONFINITE, "non-finite residual"};
            if (rel <= opts->rtol) { converged = true; break; }
            if (cycles >= opts->max_cycles) break;
            // fallback: a cycle with the learned (nonlinear) preconditioner that did not reduce the
            // true residual (by at least a relative 2^-10, so that rounding noise does not count as
            // progress) turns it off; the unpreconditioned method finishes the solve.  A fixed linear
            // preconditioner (Jacobi) is kept: its slow cycles are the restarted method's, not its own.
            const bool stalled = cycles > 0 && !(rel < prev_rel * (1.0 - 0x1p-10));
            if (use_pc && (learned || (callback && cb.nonlinear)) && stalled) {
                use_pc = false;
                fallback_cycle = cycles;
            } else if (stalled) {
                // A cycle of the restarted method that did not reduce the true residual draws a new
                // Theta for the following cycles.  Each cycle minimises the sketched residual only,
                // and after many cycles with one Theta the residual is no longer independent of it:
                // it can settle where Theta sees little of it (||Theta r|| << ||r||), and the cycles
                // then make no progress.  The new Theta is the r-th refresh of the caller's seed,
                // seed + r * 0x9E3779B97F4A7C15 (mod 2^64), with the same kind, n and k.
                ++refreshes;
                rgs_sketch ns = nullptr;
                const uint64_t seed = s->seed + (uint64_t)refreshes * 0x9E3779B97F4A7C15ull;
                const rgs_status cs = rgs_sketch_create(h, (rgs_sketch_kind)s->kind, s->n, s->k, seed, &ns);
                if (cs != RGS_OK) throw RgsError{cs, "sketch refresh: " + std::string(rgs_last_error(h))};
                fresh.reset(ns);
                obj.sk = ns;
            }
            prev_rel = rel;
            reset_cycle(&obj);
            // Arnoldi step 0: q'_0 from r, w'_1 = A M q'_0, column 0 appended and p_1 solved
            int sp = 0, pp = 0;
            step(0, sc.r, 0, nullptr, true, sp, pp);
            launch_ls(&obj, 0, sp, m >= 1, pp, true, stop_tol);
            for (int i = 1; i <= m; ++i) {
                step(i, obj.wbuf.ptr, sketch_is_df(&obj) ? 1 : 0, obj.ls.sigma + (i - 1), i < m, sp, pp);
                timer.start(2);
                launch_ls(&obj, i, sp, i < m, pp, true, stop_tol);
                timer.stop(2);
            }
            rgs_launch_hess_solve(h, obj.ls.Hr, obj.mmax, obj.ls.g, obj.ls.sigma, m, y_buf(&obj), cy_buf(&obj),
                                  h->ctl.as<int>());
            if (use_pc && learned)
                rgs_launch_sol_update(h, s->n, obj.Z.ptr, RGS_F32, obj.ldq, cy_buf(&obj), x, h->ctl.as<int>());
            else if (use_pc && cb_flex)
                rgs_launch_sol_update(h, s->n, obj.Z.ptr, ztype, obj.ldq, cy_buf(&obj), x, h->ctl.as<int>());
            else if (use_pc && callback) {                 // x += M (Q y)
                double* t = obj.pct.as<double>();
                RGS_CUDA(cudaMemsetAsync(t, 0, sizeof(double) * (size_t)s->n, h->stream));
                rgs_launch_sol_update(h, s->n, obj.Q.ptr, obj.qtype, obj.ldq, cy_buf(&obj), t, h->ctl.as<int>());
                apply_cb(t, RGS_F64, obj.Z.ptr);
                rgs_launch_add_vector(h, s->n, obj.Z.ptr, ztype, x, h->ctl.as<int>());
            } else
                rgs_launch_sol_update(h, s->n, obj.Q.ptr, obj.qtype, obj.ldq, cy_buf(&obj), x, h->ctl.as<int>(),
                                      use_pc ? dinv : nullptr);
            ++cycles;
        }
        if (trace) {
            RGS_CUDA(cudaStreamSynchronize(h->stream));
            const double nst = std::max(1, total);
            std::fprintf(stderr, "[rgs trace] rgmres, %d steps (us per step, device): update + sketch %.2f, product + "
                         "sketch %.2f, least squares %.2f\n", total, 1e3 * timer.total_ms(0) / nst,
                         1e3 * timer.total_ms(1) / nst, 1e3 * timer.total_ms(2) / nst);
            rgs_print_ls_trace(h, m + 1, rgs_ls_grid(h));
        }
        if (info) {
            info->cycles = cycles;
            info->total_steps = total;
            info->converged = converged ? 1 : 0;
            info->rel_residual = rel;
            info->fallback_cycle = fallback_cycle;
            info->sketch_refreshes = refreshes;
        }
    });
    if (info) info->status = st;
    if (st == RGS_OK && !converged) return RGS_ERR_NOT_CONVERGED;
    return st;
}

}  // extern "C"

namespace {

// After the last CGS pass of step j: ||w||, sigma_{j+1}, the Givens rotation of H(:, j), stop test.
// w = A v_j was formed from the normalised v_j = sigma_j v'_j, so H(:, j) = [sigma_t (t1 + t2)_t; ||w||].
__global__ void cgs_finish_kernel(const double* part, int np, int j, double* sigma, const double* hacc, double* cs,
                                  double* sn, double* g, double* Hr, int ldh, double stop_tol, int* ctl) {
    if (ctl[kStatusWord] != 0 || ctl[kStopWord] != 0) return;
    const int lane = threadIdx.x;
    double v = 0.0;
    for (int b = lane; b < np; b += 32) v += part[b];
    const double wn = sqrt(warp_sum(v));
    double hmax = 0.0;
    for (int t = lane; t <= j; t += 32) hmax = fmax(hmax, fabs(sigma[t] * hacc[t]));
    for (int o = 16; o > 0; o >>= 1) hmax = fmax(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
    auto hcol = [&](int t) { return t <= j ? sigma[t] * hacc[t] : wn; };
    const double res = givens_column_warp(j, hcol, cs, sn, g, Hr, ldh);
    if (lane == 0) {
        const bool breakdown = !(wn > 16.0 * 0x1p-53 * hmax);
        sigma[j + 1] = wn > 0.0 ? 1.0 / wn : 0.0;
        if (breakdown || res <= stop_tol) atomicCAS(ctl + kStopWord, 0, j + 1);
    }
}

__global__ void set_first_kernel(const double* r, const double* rnorm, int64_t n, double* v0, double* sigma,
                                 double* g) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v0[i] = r[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sigma[0] = 1.0 / rnorm[0];
        g[0] = rnorm[0];
    }
}

}  // namespace

extern "C" {

rgs_status cgs2_gmres_solve(rgs_handle h, const rgs_csr* A, const double* b, double* x, const rgmres_opts* opts,
                            rgmres_info* info) {
    if (!h || !A || !opts) return RGS_ERR_INVALID_ARG;
    if (info) {
        info->cycles = info->total_steps = info->converged = info->sell = info->sketch_refreshes = 0;
        info->status = RGS_OK;
        info->rel_residual = NAN;
    }
    bool converged = false;
    rgs_status st = guarded(h, [&] {
        check_csr(A, A->n);
        RGS_REQUIRE(b && x, "null b or x");
        RGS_REQUIRE(opts->restart >= 1 && opts->restart < 1024, "need 1 <= restart < 1024");
        const int m = opts->restart;
        const int64_t n = A->n, ldv = (n + 7) & ~(int64_t)7;
        DevBuf V, wv, gv, work;
        V.ensure(sizeof(double) * (size_t)ldv * (m + 1));
        wv.ensure(sizeof(double) * (size_t)n);
        const int mp = m + 1;
        gv.ensure(sizeof(double) * (7 * (size_t)mp + 2 + (size_t)mp * mp));
        double* sigma = gv.as<double>();
        double* cs = sigma + mp;
        double* sn = cs + mp;
        double* g = sn + mp;                    // mp + 2
        double* hacc = g + mp + 2;
        double* coef = hacc + mp;
        double* cyv = coef + mp;
        double* yv = cyv + mp;
        double* Hr = yv + mp;                   // mp x mp
        const int mdg = rgs_multidot_grid(h, n);
        work.ensure(sizeof(double) * ((size_t)n + (size_t)mdg * mp + 8 * (size_t)h->num_sms + 64));
        double* r = work.as<double>();
        double* part = r + n;                                  // multidot partials (mdg x mp)
        double* npart = part + (size_t)mdg * mp;               // norm partials
        double* val = npart + 8 * (size_t)h->num_sms;          // device scalars
        int* ctl = h->ctl.as<int>();
        h->launches = 0;
        RGS_CUDA(cudaMemsetAsync(ctl, 0, kCtlWords * sizeof(int), h->stream));
        rgs_launch_norm(h, n, b, npart, val + 1);
        double bn;
        RGS_CUDA(cudaMemcpyAsync(&bn, val + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        RGS_CUDA(cudaStreamSynchronize(h->stream));
        RGS_REQUIRE(bn > 0.0 && std::isfinite(bn), "b must be nonzero and finite");
        double stop_tol = opts->fixed_steps ? -1.0 : opts->inner_factor * opts->rtol * bn;
        const int ng = rgs_norm_grid(h, n);
        int cycles = 0, total = 0;
        double rel = NAN;
        for (;;) {
            rgs_launch_residual(h, *A, x, b, r, npart, val);
            double rn;
            int ctlv[8];
            RGS_CUDA(cudaMemcpyAsync(&rn, val, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            RGS_CUDA(cudaMemcpyAsync(ctlv, ctl, sizeof(ctlv), cudaMemcpyDeviceToHost, h->stream));
            RGS_CUDA(cudaStreamSynchronize(h->stream));
            if (ctlv[0] != 0) throw RgsError{(rgs_status)ctlv[0], "device status"};
            if (cycles > 0) total += ctlv[kStepsWord];
            rel = rn / bn;
            tighten_inner(stop_tol, cycles, ctlv[kStepsWord], m, rel, *opts);
            if (info && info->history) info->history[cycles] = rel;
            if (!std::isfinite(rel)) throw RgsError{RGS_ERR_NONFINITE, "non-finite residual"};
            if (rel <= opts->rtol) { converged = true; break; }
            if (cycles >= opts->max_cycles) break;
            RGS_CUDA(cudaMemsetAsync(ctl + kStopWord, 0, 2 * sizeof(int), h->stream));
            RGS_CUDA(cudaMemsetAsync(gv.ptr, 0, gv.bytes, h->stream));
            set_first_kernel<<<ng, 256, 0, h->stream>>>(r, val, n, V.as<double>(), sigma, g);
            RGS_CUDA(cudaGetLastError());
            for (int j = 0; j < m; ++j) {
                double* vj = V.as<double>() + (size_t)j * ldv;
                double* vn = V.as<double>() + (size_t)(j + 1) * ldv;
                // w = A v_j = sigma_j A v'_j
                rgs_launch_spmv(h, *A, nullptr, vj, RGS_F64, wv.ptr, 0, nullptr, nullptr, ctl, sigma + j);
                rgs_launch_cgs_pass(h, n, V.as<double>(), ldv, j + 1, sigma, wv.as<double>(), part, coef, hacc, 0, ctl);
                rgs_launch_cgs_update(h, n, V.as<double>(), ldv, j + 1, coef, wv.as<double>(), nullptr, nullptr, ctl);
                rgs_launch_cgs_pass(h, n, V.as<double>(), ldv, j + 1, sigma, wv.as<double>(), part, coef, hacc, 1, ctl);
                rgs_launch_cgs_update(h, n, V.as<double>(), ldv, j + 1, coef, wv.as<double>(), vn, npart, ctl);
                cgs_finish_kernel<<<1, 32, 0, h->stream>>>(npart, ng, j, sigma, hacc, cs, sn, g, Hr, mp, stop_tol, ctl);
                RGS_CUDA(cudaGetLastError());
            }
            rgs_launch_hess_solve(h, Hr, mp, g, sigma, m, yv, cyv, ctl);
            rgs_launch_sol_update(h, n, V.ptr, RGS_F64, ldv, cyv, x, ctl);
            ++cycles;
        }
        if (info) {
            info->cycles = cycles;
            info->total_steps = total;
            info->converged = converged ? 1 : 0;
            info->rel_residual = rel;
        }
    });
    if (info) info->status = st;
    if (st == RGS_OK && !converged) return RGS_ERR_NOT_CONVERGED;
    return st;
}

rgs_status rgmres_set_preconditioner(rgs_handle h, rgs_precond_kind kind, const void* params, int32_t flexible) {
    if (!h) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_REQUIRE(kind == RGS_PRECOND_NONE || kind == RGS_PRECOND_JACOBI || kind == RGS_PRECOND_LEARNED_CONV ||
                        kind == RGS_PRECOND_CALLBACK,
                    "unknown preconditioner kind");
        rgs_callback_precond cb{};
        if (kind == RGS_PRECOND_CALLBACK) {
            RGS_REQUIRE(params != nullptr, "the callback preconditioner needs rgs_callback_precond parameters");
            cb = *static_cast<const rgs_callback_precond*>(params);
            RGS_REQUIRE(cb.apply != nullptr, "null apply function");
            RGS_REQUIRE(flexible || !cb.nonlinear, "a nonlinear preconditioner needs flexible GMRES (flexible = 1)");
        }
        if (kind == RGS_PRECOND_LEARNED_CONV) {
            RGS_REQUIRE(params != nullptr, "the learned preconditioner needs rgs_learned_precond parameters");
            RGS_REQUIRE(flexible, "a nonlinear preconditioner needs flexible GMRES (flexible = 1)");
            const rgs_learned_precond* lp = static_cast<const rgs_learned_precond*>(params);
            RGS_REQUIRE(lp->net != nullptr && lp->logkappa != nullptr, "null network or field");
            h->precond_net = lp->net;
            h->precond_field = lp->logkappa;
        } else {
            h->precond_net = nullptr;
            h->precond_field = nullptr;
        }
        h->precond_cb = cb;
        h->precond_kind = kind;
        h->precond_flexible = flexible;
    });
}

rgs_status rgs_csr_residual(rgs_handle h, const rgs_csr* A, const double* x, const double* b, double* r,
                            double* rnorm) {
    if (!h) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_REQUIRE(A != nullptr, "null CSR");
        check_csr(A, A->n);
        RGS_REQUIRE(A->n >= 1 && x && b && r, "need n >= 1 and x, b, r");
        RGS_REQUIRE(r != x, "r and x must not alias");
        const int grid = rgs_norm_grid(h, A->n);
        h->work.ensure(sizeof(double) * ((size_t)grid + 1));
        double* part = h->work.as<double>();
        rgs_launch_residual(h, *A, x, b, r, part, part + grid);
        if (rnorm) {
            RGS_CUDA(cudaMemcpyAsync(rnorm, part + grid, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            RGS_CUDA(cudaStreamSynchronize(h->stream));
        }
    });
}

rgs_status rgs_csr_matvec(rgs_handle h, const rgs_csr* A, const double* x, double* y) {
    if (!h) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_REQUIRE(A != nullptr, "null CSR");
        check_csr(A, A->n);
        RGS_REQUIRE(A->n == 0 || (x && y), "null x or y");
        RGS_REQUIRE(x != y, "x and y must not alias");
        if (A->n == 0) return;
        rgs_launch_spmv(h, *A, nullptr, x, RGS_F64, y, 0, nullptr, nullptr, nullptr);
    });
}



}  // extern "C"
