// C entry points of librgs: handle, sketches, and the RGS QR driver (Alg. 2).
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

using namespace rgsdev;

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

__global__ void srht_signbits_kernel(uint32_t* bits, int64_t nblocks, uint32_t key0, uint32_t key1) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    uint32_t c[4] = {(uint32_t)b, 0u, 0u, 1u};
    philox4x32_10(c, key0, key1);
    for (int t = 0; t < 4; ++t) bits[4 * b + t] = c[t];
}

// Q(:, j) *= qscale[j], rounded back to the storage type (Step 7 applied at the end).
template <typename TQ>
__global__ void scale_columns_kernel(TQ* Q, int64_t n, int m, int64_t ldq, const double* sigma) {
    const int j = blockIdx.y;
    const double s = sigma[j];
    TQ* col = Q + (int64_t)j * ldq;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (sizeof(TQ) == 2) col[r] = __float2bfloat16_rn((float)((double)__bfloat162float(col[r]) * s));
        else col[r] = (TQ)((double)col[r] * s);
    }
}

void scale_columns(rgs_context* ctx, void* Q, int qtype, int64_t n, int m, int64_t ldq, const double* sigma) {
    const int gx = (int)std::min<int64_t>((n + 255) / 256, 64);
    dim3 grid(gx, m);
    if (qtype == RGS_F64) scale_columns_kernel<double><<<grid, 256, 0, ctx->stream>>>((double*)Q, n, m, ldq, sigma);
    else if (qtype == RGS_F32) scale_columns_kernel<float><<<grid, 256, 0, ctx->stream>>>((float*)Q, n, m, ldq, sigma);
    else scale_columns_kernel<__nv_bfloat16><<<grid, 256, 0, ctx->stream>>>((__nv_bfloat16*)Q, n, m, ldq, sigma);
    RGS_CUDA(cudaGetLastError());
    ctx->launches++;
}

size_t dtype_size(int t) { return t == RGS_F64 ? 8 : (t == RGS_F32 ? 4 : 2); }

bool is_host_pointer(const void* p) { return rgs_is_host_pointer(p); }

void reset_ctl(rgs_context* ctx) {
    RGS_CUDA(cudaMemsetAsync(ctx->ctl.ptr, 0, kCtlWords * sizeof(int), ctx->stream));
}

// Y (k x ncols) = Theta X, in column batches whose partial sketches fit a fixed budget.
// fine: transform sums 0 FP64, 1 double-float, 2 FP32 (SRHT).
void sketch_block(rgs_context* ctx, const rgs_sketch_obj* sk, int ncols, const double* X, int64_t ldx, double* Y,
                  int64_t ldy, int df = 0) {
    const int k = sk->k;
    const double scale = sk->kind == RGS_SKETCH_SRHT ? 1.0 / std::sqrt((double)k) : 1.0;
    const size_t budget = (size_t)256 << 20;
    int batch = std::min(ncols, kMaxGridY);
    while (batch > 1 && (size_t)batch * rgs_update_nparts(ctx, sk, sk->n, batch) * k * 8 > budget) batch = (batch + 1) / 2;
    for (int c0 = 0; c0 < ncols; c0 += batch) {
        const int nc = std::min(batch, ncols - c0);
        const int np = rgs_update_nparts(ctx, sk, sk->n, nc);
        ctx->partials.ensure((size_t)nc * np * k * 8);
        UpdateLaunch L{};
        L.n = sk->n;
        L.ncols = 0;
        L.qtype = RGS_F64;
        L.w = X + (int64_t)c0 * ldx;
        L.ldw = ldx;
        L.wcols = nc;
        L.df_sketch = df;
        int nparts = 0;
        rgs_launch_update_sketch(ctx, sk, L, ctx->partials.as<double>(), &nparts, nullptr);
        rgs_launch_reduce_partials(ctx, ctx->partials.as<double>(), nparts, k, nc, scale, Y + (int64_t)c0 * ldy, ldy,
                                   df != 0 && sk->kind == RGS_SKETCH_SRHT);
    }
}

}  // namespace

void rgs_sketch_columns(rgs_context* ctx, const rgs_sketch_obj* sk, int ncols, const double* X, int64_t ldx,
                        double* Y, int64_t ldy) {
    sketch_block(ctx, sk, ncols, X, ldx, Y, ldy, false);
}

bool rgs_is_host_pointer(const void* p) {
    if (p == nullptr) return false;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return attr.type == cudaMemoryTypeHost || attr.type == cudaMemoryTypeUnregistered;
}

// RGS_TRACE summary of the least-squares launches in microseconds, as means over the launches of
// each range of 50 columns: the spread of the CTAs' start times; per phase the median CTA's work
// (from leaving the previous barrier to arriving at the next), how long after the median CTA the
// last one arrived, and the barrier's own latency (from the last arrival to the median
// departure); the last phase up to the last CTA's end; the launch's first start to last end.
void rgs_print_ls_trace(rgs_context* h, int m, int grid) {
    const size_t stride = (size_t)grid * kLsTraceSlots;
    std::vector<unsigned long long> t(stride * (size_t)m);
    RGS_CUDA(cudaMemcpy(t.data(), h->trace.ptr, t.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    constexpr int kBucket = 50;
    const int nbk = (m + kBucket - 1) / kBucket;
    struct Acc {
        double start = 0, work[4] = {0}, skew[4] = {0}, lat[4] = {0}, tail = 0, total = 0, psum_med = 0, psum_max = 0;
        double item[4] = {0};   // first item: start -> sums, -> barrier, -> warp 0's totals, -> end of the items
        int n = 0, nq[4] = {0};
    };
    std::vector<Acc> acc(nbk);
    auto median = [](std::vector<double> v) {
        std::nth_element(v.begin(), v.begin() + v.size() / 2, v.end());
        return v[v.size() / 2];
    };
    std::vector<double> a(grid), d(grid), prev(grid), w(grid);
    for (int i = 0; i < m; ++i) {
        const unsigned long long* ti = t.data() + stride * (size_t)i;
        auto at = [&](int b, int slot) { return ti[(size_t)b * kLsTraceSlots + slot]; };
        if (at(0, 0) == 0) continue;                               // not launched (early stop)
        Acc& c = acc[i / kBucket];
        ++c.n;
        unsigned long long t0 = at(0, 0), t1 = at(0, 0), e1 = 0;
        for (int b = 0; b < grid; ++b) {
            t0 = std::min(t0, at(b, 0));
            t1 = std::max(t1, at(b, 0));
            e1 = std::max(e1, at(b, 9));
        }
        c.start += (double)(t1 - t0) * 1e-3;
        for (int b = 0; b < grid; ++b) {
            prev[b] = (double)(at(b, 0) - t0);
            w[b] = (double)(at(b, 10) - at(b, 0));                 // phase 0's partial sums
        }
        c.psum_med += median(w) * 1e-3;
        c.psum_max += *std::max_element(w.begin(), w.end()) * 1e-3;
        for (int q = 0; q < 3; ++q) {                              // inside the first item (CTAs with one)
            std::vector<double> u;
            for (int b = 0; b < grid; ++b) {
                const unsigned long long s1 = at(b, 11 + q), s0 = q == 0 ? at(b, 0) : at(b, 10 + q);
                if (s1 != 0 && s0 != 0 && s1 >= s0) u.push_back((double)(s1 - s0));
            }
            if (!u.empty()) c.item[q] += median(u) * 1e-3;
        }
        {
            std::vector<double> u;
            for (int b = 0; b < grid; ++b)
                if (at(b, 13) != 0 && at(b, 10) >= at(b, 13)) u.push_back((double)(at(b, 10) - at(b, 13)));
            if (!u.empty()) c.item[3] += median(u) * 1e-3;
        }
        for (int q = 0; q < 4; ++q) {
            if (at(0, 1 + 2 * q) == 0) break;                      // this launch had fewer barriers
            for (int b = 0; b < grid; ++b) {
                a[b] = (double)(at(b, 1 + 2 * q) - t0);
                d[b] = (double)(at(b, 2 + 2 * q) - t0);
                w[b] = a[b] - prev[b];
            }
            const double amax = *std::max_element(a.begin(), a.end());
            c.work[q] += median(w) * 1e-3;
            c.skew[q] += (amax - median(a)) * 1e-3;
            c.lat[q] += (median(d) - amax) * 1e-3;
            ++c.nq[q];
            prev = d;
        }
        c.tail += ((double)(e1 - t0) - median(prev)) * 1e-3;
        c.total += (double)(e1 - t0) * 1e-3;
    }
    for (int bk = 0; bk < nbk; ++bk) {
        const Acc& c = acc[bk];
        if (c.n == 0) continue;
        std::fprintf(stderr, "[rgs trace] least squares, columns [%d,%d), %d CTAs (us): start spread %.2f; "
                     "partial sums median %.2f, max %.2f (first item: sums %.2f, barrier %.2f, totals %.2f, rest %.2f)",
                     bk * kBucket, std::min(m, (bk + 1) * kBucket), grid, c.start / c.n, c.psum_med / c.n,
                     c.psum_max / c.n, c.item[0] / c.n, c.item[1] / c.n, c.item[2] / c.n, c.item[3] / c.n);
        for (int q = 0; q < 4; ++q)
            if (c.nq[q] > 0)
                std::fprintf(stderr, "; phase %d work %.2f, last arrival +%.2f, barrier %.2f", q, c.work[q] / c.nq[q],
                             c.skew[q] / c.nq[q], c.lat[q] / c.nq[q]);
        std::fprintf(stderr, "; last phase %.2f; launch %.2f\n", c.tail / c.n, c.total / c.n);
    }
}

extern "C" {

const char* rgs_status_string(rgs_status s) {
    switch (s) {
        case RGS_OK: return "ok";
        case RGS_ERR_INVALID_ARG: return "invalid argument";
        case RGS_ERR_CUDA: return "CUDA error";
        case RGS_ERR_ALLOC: return "allocation failed";
        case RGS_ERR_BREAKDOWN: return "breakdown (r_ii vanished)";
        case RGS_ERR_NOT_CONVERGED: return "not converged";
        case RGS_ERR_TIMEOUT: return "device barrier timeout";
        case RGS_ERR_NONFINITE: return "non-finite value";
        case RGS_ERR_NOT_IMPLEMENTED: return "not implemented";
        case RGS_ERR_CERT_FAILED: return "no embedding certificate (omega_bar >= 1)";
        case RGS_ERR_CALLBACK: return "the preconditioner callback failed";
    }
    return "unknown status";
}

const char* rgs_last_error(rgs_handle h) { return h ? h->last_error.c_str() : "null handle"; }

rgs_status rgs_create(rgs_handle* out, void* stream) {
    if (!out) return RGS_ERR_INVALID_ARG;
    *out = nullptr;
    rgs_context* ctx = new (std::nothrow) rgs_context();
    if (!ctx) return RGS_ERR_ALLOC;
    rgs_status st = guarded(ctx, [&] {
        RGS_CUDA(cudaGetDevice(&ctx->device));
        RGS_CUDA(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
        int coop = 0;
        RGS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device));
        RGS_REQUIRE(coop, "device does not support cooperative launches");
        ctx->stream = (cudaStream_t)stream;
        ctx->ctl.ensure(kCtlAlloc * sizeof(int));
        RGS_CUDA(cudaMemset(ctx->ctl.ptr, 0, kCtlAlloc * sizeof(int)));
        ctx->ls_blocks = rgs_ls_max_blocks(ctx->num_sms);
        const char* pdl = std::getenv("RGS_PDL");
        ctx->pdl = (pdl != nullptr && pdl[0] == '0') ? 0 : 1;
        rgs_noalloc_reserve(ctx->device);
    });
    if (st != RGS_OK) {
        delete ctx;
        return st;
    }
    *out = ctx;
    return RGS_OK;
}

rgs_status rgs_destroy(rgs_handle h) {
    if (!h) return RGS_ERR_INVALID_ARG;
    cudaStreamSynchronize(h->stream);
    delete h;
    return RGS_OK;
}

rgs_status rgs_set_wait_budget(rgs_handle h, int64_t cycles) {
    if (!h) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        const long long v = cycles > 0 ? (long long)cycles : 0;
        RGS_CUDA(cudaMemcpyAsync(h->ctl.as<int>() + kBudgetWord, &v, sizeof(v), cudaMemcpyHostToDevice, h->stream));
        RGS_CUDA(cudaStreamSynchronize(h->stream));
    });
}

rgs_status rgs_set_stream(rgs_handle h, void* stream) {
    if (!h) return RGS_ERR_INVALID_ARG;
    h->stream = (cudaStream_t)stream;
    return RGS_OK;
}

rgs_status rgs_sketch_create(rgs_handle h, rgs_sketch_kind kind, int64_t n, int32_t k, uint64_t seed,
                             rgs_sketch* out) {
    if (!h || !out) return RGS_ERR_INVALID_ARG;
    *out = nullptr;
    rgs_sketch_obj* sk = new (std::nothrow) rgs_sketch_obj();
    if (!sk) return RGS_ERR_ALLOC;
    rgs_status st = guarded(h, [&] {
        RGS_REQUIRE(kind == RGS_SKETCH_GAUSSIAN || kind == RGS_SKETCH_SRHT, "unknown sketch kind");
        RGS_REQUIRE(n >= 1 && n < ((int64_t)1 << 31), "n must be in [1, 2^31)");
        RGS_REQUIRE(k >= 1, "k must be >= 1");
        sk->h = h;
        sk->kind = kind;
        sk->n = n;
        sk->k = k;
        sk->seed = seed;
        sk->s = 1;
        while (sk->s < n) sk->s *= 2;
        const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
        if (kind == RGS_SKETCH_GAUSSIAN) {
            sk->theta.ensure(sizeof(double) * (size_t)k * (size_t)n);
            rgs_launch_gaussian_theta(h, sk->theta.as<double>(), k, n, seed);
        } else {
            RGS_REQUIRE(k <= sk->s, "SRHT needs k <= s (the power of two >= n)");
            const int64_t nblocks = (n + 127) / 128;
            sk->signbits.ensure(sizeof(uint32_t) * 4 * (size_t)nblocks);
            srht_signbits_kernel<<<(unsigned)((nblocks + 255) / 256), 256, 0, h->stream>>>(sk->signbits.as<uint32_t>(),
                                                                                           nblocks, key0, key1);
            RGS_CUDA(cudaGetLastError());
            // uniform sample without replacement: the k smallest (key, index) pairs
            std::vector<std::pair<uint64_t, int64_t>> keys((size_t)sk->s);
            for (int64_t c = 0; c < sk->s; ++c) {
                uint32_t ctr[4] = {(uint32_t)c, 0u, 0u, 2u};
                philox4x32_10(ctr, key0, key1);
                keys[(size_t)c] = {((uint64_t)ctr[0] << 32) | ctr[1], c};
            }
            std::nth_element(keys.begin(), keys.begin() + (k - 1), keys.end());
            std::vector<int32_t> rows((size_t)k);
            for (int j = 0; j < k; ++j) rows[(size_t)j] = (int32_t)keys[(size_t)j].second;
            std::sort(rows.begin(), rows.end());
            sk->rows.ensure(sizeof(int32_t) * (size_t)k);
            RGS_CUDA(cudaMemcpyAsync(sk->rows.ptr, rows.data(), sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice,
                                     h->stream));
            RGS_CUDA(cudaStreamSynchronize(h->stream));
        }
    });
    if (st != RGS_OK) {
        delete sk;
        return st;
    }
    *out = sk;
    return RGS_OK;
}

// The sketch outlives nothing it points to: its device tables are released with cudaFree
// (which waits for work in flight) and the handle it was created on is not touched, so it
// may be destroyed before or after that handle.
rgs_status rgs_sketch_destroy(rgs_sketch s) {
    if (!s) return RGS_ERR_INVALID_ARG;
    delete s;
    return RGS_OK;
}

rgs_status rgs_sketch_apply(rgs_handle h, rgs_sketch s, int32_t ncols, const double* X, int64_t ldx, double* Y,
                            int64_t ldy) {
    if (!h || !s) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_REQUIRE(ncols >= 0, "ncols must be >= 0");
        RGS_REQUIRE(ncols == 0 || (X && Y), "null X or Y");
        RGS_REQUIRE(ldx >= s->n && ldy >= s->k, "leading dimension too small");
        RGS_REQUIRE(ncols == 0 || (!is_host_pointer(X) && !is_host_pointer(Y)), "X and Y must be device pointers");
        if (ncols == 0) return;
        sketch_block(h, s, ncols, X, ldx, Y, ldy);
    });
}

rgs_status rgs_qr(rgs_handle h, rgs_sketch s, int64_t n, int32_t m, const double* W, int64_t ldw, void* Q,
                  rgs_dtype qtype, int64_t ldq, double* qscale, double* R, int64_t ldr, double* S, int64_t lds,
                  int32_t flags, rgs_qr_info* info) {
    if (!h || !s) return RGS_ERR_INVALID_ARG;
    if (info) {
        info->delta = NAN;
        info->delta_tilde = NAN;
        info->breakdown_col = -1;
        info->launches = 0;
        info->sketch_ms = info->update_ms = info->ls_ms = NAN;
    }
    return guarded(h, [&] {
        RGS_REQUIRE(qtype == RGS_F64 || qtype == RGS_F32 || qtype == RGS_BF16, "unknown qtype");
        RGS_REQUIRE(n == s->n, "n differs from the sketch's n");
        RGS_REQUIRE(!(flags & RGS_LS_RICHARDSON) || qtype == RGS_F64 || (flags & (RGS_FP64_LS | RGS_FP64_FINE)),
                    "RGS_LS_RICHARDSON needs FP64 least squares (an FP64 basis, RGS_FP64_LS or RGS_FP64_FINE)");
        RGS_REQUIRE(!(flags & RGS_FP32_FINE) || (qtype != RGS_F64 && s->kind == RGS_SKETCH_SRHT &&
                                                 !(flags & (RGS_FP64_FINE | RGS_FP64_LS))),
                    "RGS_FP32_FINE needs an FP32 / BF16 basis, an SRHT sketch and no FP64 fine flag");
        RGS_REQUIRE(m >= 1 && m <= s->k, "need 1 <= m <= k (Alg. 2 assumes m <= k)");
        RGS_REQUIRE(m <= n, "need m <= n");
        RGS_REQUIRE(W && Q && R, "null W, Q or R");
        RGS_REQUIRE(ldw >= n && ldq >= n && ldr >= m, "leading dimension too small");
        RGS_REQUIRE(!S || lds >= s->k, "lds must be >= k");
        const int k = s->k;
        const size_t esz = dtype_size(qtype);
        cudaStream_t st = h->stream;

        // host pointers are staged through device memory
        const bool host = is_host_pointer(W);
        RGS_REQUIRE(host == is_host_pointer(Q) && host == is_host_pointer(R) && (!S || host == is_host_pointer(S)) &&
                        (!qscale || host == is_host_pointer(qscale)),
                    "W, Q, R, S, qscale must be all host or all device pointers");
        const double* dW = W;
        void* dQ = Q;
        double* dR = R;
        int64_t dldw = ldw, dldq = ldq, dldr = ldr;
        // With the SRHT, column i of W is needed only from the update pass of column i - 1, and
        // (with qscale) q'_i is final after its own pass: host copies then run in column chunks on
        // a copy stream, overlapped with the factorization, ordered by events.
        const bool pipelined = host && s->kind == RGS_SKETCH_SRHT;
        const int CB = 8;                                       // columns per copy chunk
        const int nchunks = (m + CB - 1) / CB;
        std::vector<cudaEvent_t> wready, qdone;
        struct EventList {
            std::vector<cudaEvent_t>* v[2];
            ~EventList() {
                for (auto* l : v)
                    for (auto e : *l) cudaEventDestroy(e);
            }
        } event_guard{{&wready, &qdone}};
        if (host) {
            const size_t wb = sizeof(double) * (size_t)n * m, qb = esz * (size_t)n * m, rb = sizeof(double) * (size_t)m * m;
            h->scratch.ensure(wb + qb + rb + 256);
            char* base = h->scratch.as<char>();
            double* sW = reinterpret_cast<double*>(base);
            dQ = base + wb;
            dR = reinterpret_cast<double*>(base + wb + qb);
            if (pipelined) {
                if (!h->copy_stream) RGS_CUDA(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
                // a previous call that failed midway may have left copies in flight on the copy
                // stream: the bound stream waits for them before the staging is written again
                cudaEvent_t prev_ev;
                RGS_CUDA(cudaEventCreateWithFlags(&prev_ev, cudaEventDisableTiming));
                qdone.push_back(prev_ev);                        // (destroyed with the others)
                RGS_CUDA(cudaEventRecord(prev_ev, h->copy_stream));
                RGS_CUDA(cudaStreamWaitEvent(st, prev_ev, 0));
                cudaEvent_t start_ev;
                RGS_CUDA(cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming));
                wready.push_back(start_ev);                      // (destroyed with the others)
                RGS_CUDA(cudaEventRecord(start_ev, st));         // earlier work on the staging is done
                RGS_CUDA(cudaStreamWaitEvent(h->copy_stream, start_ev, 0));
                for (int c = 0; c < nchunks; ++c) {
                    const int c0 = c * CB, cols = std::min(CB, m - c0);
                    RGS_CUDA(cudaMemcpy2DAsync(sW + (size_t)c0 * n, sizeof(double) * n, W + (size_t)c0 * ldw,
                                               sizeof(double) * ldw, sizeof(double) * n, cols, cudaMemcpyHostToDevice,
                                               h->copy_stream));
                    cudaEvent_t e;
                    RGS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                    wready.push_back(e);
                    RGS_CUDA(cudaEventRecord(e, h->copy_stream));
                }
            } else {
                RGS_CUDA(cudaMemcpy2DAsync(sW, sizeof(double) * n, W, sizeof(double) * ldw, sizeof(double) * n, m,
                                           cudaMemcpyHostToDevice, st));
            }
            dW = sW;
            dldw = n;
            dldq = n;
            dldr = m;
        }
        // chunk c of W is on the device once wready[1 + c] has completed
        int w_waited = -1;
        auto need_w = [&](int col) {
            if (!pipelined) return;
            const int c = std::min(col, m - 1) / CB;
            while (w_waited < c) {
                ++w_waited;
                RGS_CUDA(cudaStreamWaitEvent(st, wready[1 + w_waited], 0));
            }
        };
        const bool early_q = pipelined && qscale != nullptr;   // Q' columns final as they are written

        // workspaces: Householder engine, P = Theta W, partial sketches, certificates
        LSState ls{};
        const bool up = (flags & RGS_FP32_FINE) != 0;     // unique precision: fine arithmetic in FP32
        rgs_ls_alloc(h->lsbuf, k, m, h->num_sms, h->num_sms * kUpdMaxBlocksPerSm,
                     up ? 2 : (qtype != RGS_F64 && !(flags & (RGS_FP64_FINE | RGS_FP64_LS)) ? 1 : 0), &ls);
        ls.ctl = h->ctl.as<int>();
        ls.R = dR;
        ls.ldr = dldr;
        h->work.ensure(sizeof(double) * ((size_t)k * m + 3 * (size_t)m + 8));
        double* P = h->work.as<double>();
        double* certw = P + (size_t)k * m;
        double* certo = certw + 3 * (size_t)m;
        const int np1 = rgs_update_nparts(h, s, n, 1);
        // SRHT: step 1 of column i + 1 is sketched in the same pass as steps 3-4 of column i
        const bool fused_p = s->kind == RGS_SKETCH_SRHT;
        h->partials.ensure(sizeof(double) * (size_t)np1 * k * (fused_p ? 2 : 1));

        PhaseTimer timer(h, (flags & RGS_QR_TIMINGS) != 0);
        // RGS_TRACE=1 in the environment: per-phase device timestamps of the least-squares kernel
        const bool trace = std::getenv("RGS_TRACE") != nullptr;
        const int ls_grid = rgs_ls_grid(h);
        const size_t tstride = (size_t)ls_grid * kLsTraceSlots;
        if (trace) {
            h->trace.ensure(sizeof(unsigned long long) * tstride * (size_t)m);
            RGS_CUDA(cudaMemsetAsync(h->trace.ptr, 0, sizeof(unsigned long long) * tstride * (size_t)m, st));
        }
        h->launches = 0;
        reset_ctl(h);
        rgs_ls_reset(h, ls);
        RGS_CUDA(cudaMemset2DAsync(dR, sizeof(double) * dldr, 0, sizeof(double) * m, m, st));

        // step 1: P = Theta W in one pass over W (Gaussian), or only p_1 (SRHT; the other
        // columns are sketched inside the update passes)
        timer.start(0);
        // transform sums: FP32 (unique precision), double-float (FP32 / BF16 bases), else FP64
        const int df = up ? 2 : (qtype != RGS_F64 && !(flags & RGS_FP64_FINE) ? 1 : 0);
        need_w(fused_p ? 0 : m - 1);
        sketch_block(h, s, fused_p ? 1 : m, dW, dldw, P, k, df);
        timer.stop(0);
        h->partials.ensure(sizeof(double) * (size_t)np1 * k * (fused_p ? 2 : 1));

        const double s_scale = s->kind == RGS_SKETCH_SRHT ? 1.0 / std::sqrt((double)k) : 1.0;
        for (int i = 0; i < m; ++i) {
            UpdateLaunch L{};
            L.n = n;
            L.ncols = i;
            L.Q = dQ;
            L.ldq = dldq;
            L.qtype = qtype;
            L.w = dW + (int64_t)i * dldw;
            L.ldw = dldw;
            L.wcols = 1;
            L.coef = ls.coef;
            L.qout = static_cast<char*>(dQ) + esz * (size_t)i * dldq;
            L.df_sketch = df;
            L.w_next = (fused_p && i + 1 < m) ? dW + (int64_t)(i + 1) * dldw : nullptr;
            int nparts = 0;
            need_w(i + 1);
            timer.start(1);
            rgs_launch_update_sketch(h, s, L, h->partials.as<double>(), &nparts, ls.ctl);   // steps 3, 4
            timer.stop(1);
            if (early_q && ((i + 1) % CB == 0 || i + 1 == m)) {
                // chunk of q' columns complete: copy it back while the factorization continues
                const int c0 = (i / CB) * CB, cols = i + 1 - c0;
                cudaEvent_t e;
                RGS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                qdone.push_back(e);
                RGS_CUDA(cudaEventRecord(e, st));
                RGS_CUDA(cudaStreamWaitEvent(h->copy_stream, e, 0));
                RGS_CUDA(cudaMemcpy2DAsync(static_cast<char*>(Q) + esz * (size_t)c0 * ldq, esz * ldq,
                                           static_cast<char*>(dQ) + esz * (size_t)c0 * dldq, esz * dldq, esz * n, cols,
                                           cudaMemcpyDeviceToHost, h->copy_stream));
            }
            LSStep a{};
            a.i = i;
            a.append = 1;                                      // steps 5, 6 (+ append to the QR of S)
            a.s_part = h->partials.as<double>();
            a.s_nparts = nparts;
            a.s_scale = s_scale;
            a.s_df = (df != 0 && s->kind == RGS_SKETCH_SRHT) ? 1 : 0;
            a.solve = (i + 1 < m) ? 1 : 0;                     // step 2 of the next column
            a.xcol = i + 1;
            if (fused_p) {
                a.p_part = h->partials.as<double>() + (size_t)nparts * k;
                a.p_nparts = nparts;
                a.p_df = a.s_df;
                a.p_scale = s_scale;
                a.p_store = P + (size_t)(i + 1) * k;
            } else {
                a.p_vec = P + (size_t)(i + 1) * k;
                a.p_scale = 1.0;
            }
            a.pnorm_idx = i + 1;
            a.rich = (flags & RGS_LS_RICHARDSON) ? 1 : 0;
            a.trace = trace ? h->trace.as<unsigned long long>() + tstride * (size_t)i : nullptr;
            timer.start(2);
            rgs_launch_ls(h, ls, a);
            timer.stop(2);
        }

        if (qscale) {
            RGS_CUDA(cudaMemcpyAsync(qscale, ls.sigma, sizeof(double) * m, host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
        } else {
            scale_columns(h, dQ, qtype, n, m, dldq, ls.sigma);
        }
        if (S) {
            RGS_CUDA(cudaMemcpy2DAsync(S, sizeof(double) * lds, ls.S, sizeof(double) * k, sizeof(double) * k, m,
                                       host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
        }
        const bool certs = !(flags & RGS_QR_NO_CERTIFICATES);
        if (certs) rgs_launch_certificates(h, ls.S, k, m, dR, dldr, P, certo, certw);
        if (host) {
            if (!early_q)
                RGS_CUDA(cudaMemcpy2DAsync(Q, esz * ldq, dQ, esz * dldq, esz * n, m, cudaMemcpyDeviceToHost, st));
            RGS_CUDA(cudaMemcpy2DAsync(R, sizeof(double) * ldr, dR, sizeof(double) * dldr, sizeof(double) * m, m,
                                       cudaMemcpyDeviceToHost, st));
        }
        if (pipelined) {
            // every copy on the copy stream (the last Q' chunks) is done before the call returns,
            // and later work on the bound stream waits for it
            cudaEvent_t e;
            RGS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            qdone.push_back(e);
            RGS_CUDA(cudaEventRecord(e, h->copy_stream));
            RGS_CUDA(cudaStreamWaitEvent(st, e, 0));
        }
        int ctl[2] = {0, 0};
        double cert[2] = {NAN, NAN};
        RGS_CUDA(cudaMemcpyAsync(ctl, h->ctl.ptr, sizeof(ctl), cudaMemcpyDeviceToHost, st));
        if (certs) RGS_CUDA(cudaMemcpyAsync(cert, certo, sizeof(cert), cudaMemcpyDeviceToHost, st));
        RGS_CUDA(cudaStreamSynchronize(st));
        if (info) {
            info->delta = cert[0];
            info->delta_tilde = cert[1];
            info->breakdown_col = ctl[0] == RGS_ERR_BREAKDOWN ? ctl[1] : -1;
            info->launches = h->launches;
            if (timer.on) {
                info->sketch_ms = timer.total_ms(0);
                info->update_ms = timer.total_ms(1);
                info->ls_ms = timer.total_ms(2);
            }
        }
        if (trace) rgs_print_ls_trace(h, m, ls_grid);
        if (ctl[0] != 0)
            throw RgsError{(rgs_status)ctl[0], std::string("device status ") + rgs_status_string((rgs_status)ctl[0]) +
                                                   " at column " + std::to_string(ctl[1])};
    });
}

}  // extern "C"
