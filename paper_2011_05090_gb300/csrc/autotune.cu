// Launch-shape tuning: the handle's tunable launch parameters, and two autotuners that time the
// candidates on the caller's own problem shape and keep the fastest on the handle.
//   - the fused update / sketch pass (steps 3-4, Alg. 2): CTAs per SM, which also sets how many
//     partial sketches the least-squares step reduces;
//   - the batched solver: CTAs per SM of the persistent grid and the work per CTA below which a
//     team gets no extra CTA (more CTAs per team shorten its steps but add team barriers).
// Every candidate computes the same quantities; only the grouping of partial sums changes.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

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
    } catch (...) {
        if (h) h->last_error = "unexpected exception";
        return RGS_ERR_INVALID_ARG;
    }
}

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    Events() {
        RGS_CUDA(cudaEventCreate(&a));
        RGS_CUDA(cudaEventCreate(&b));
    }
    ~Events() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

void fill_tuning(const rgs_context* h, rgs_tuning* t) {
    t->upd_blocks_per_sm = h->upd_blocks_per_sm;
    t->batch_blocks_per_sm = h->batch_blocks_per_sm;
    t->batch_min_team_work = h->batch_min_team_work;
    t->ls_blocks = h->ls_blocks_tuned;
    t->batch_rows_per_thread = h->batch_rr;
}

__global__ void fill_kernel(double* q, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        q[i] = (double)((i * 2654435761u) & 1023) * (1.0 / 1024.0);
}

}  // namespace

extern "C" {

rgs_status rgs_get_tuning(rgs_handle h, rgs_tuning* out) {
    if (!h || !out) return RGS_ERR_INVALID_ARG;
    fill_tuning(h, out);
    return RGS_OK;
}

rgs_status rgs_set_tuning(rgs_handle h, const rgs_tuning* t) {
    if (!h || !t) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_REQUIRE(t->upd_blocks_per_sm >= 1 && t->upd_blocks_per_sm <= kUpdMaxBlocksPerSm,
                    "upd_blocks_per_sm must be in [1, 4]");
        RGS_REQUIRE(t->batch_blocks_per_sm >= 0 && t->batch_blocks_per_sm <= 4, "batch_blocks_per_sm must be in [0, 4]");
        RGS_REQUIRE(t->batch_min_team_work > 0.0, "batch_min_team_work must be positive");
        RGS_REQUIRE(t->ls_blocks >= 0 && t->ls_blocks <= h->num_sms, "ls_blocks must be in [0, SMs]");
        RGS_REQUIRE(t->batch_rows_per_thread == 0 || t->batch_rows_per_thread == 2 || t->batch_rows_per_thread == 4,
                    "batch_rows_per_thread must be 0 (4), 2 or 4");
        h->ls_blocks_tuned = t->ls_blocks;
        h->batch_rr = t->batch_rows_per_thread == 0 ? 4 : t->batch_rows_per_thread;
        h->upd_blocks_per_sm = t->upd_blocks_per_sm;
        h->batch_blocks_per_sm = t->batch_blocks_per_sm;
        h->batch_min_team_work = t->batch_min_team_work;
    });
}

rgs_status rgs_autotune_update(rgs_handle h, rgs_sketch s, int32_t ncols, rgs_dtype qtype, rgs_tuning* out,
                               float* ms) {
    if (!h || !s) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_REQUIRE(s->kind == RGS_SKETCH_SRHT, "the update pass is tuned with an SRHT sketch");
        RGS_REQUIRE(ncols >= 1, "ncols must be >= 1");
        RGS_REQUIRE(qtype == RGS_F64 || qtype == RGS_F32 || qtype == RGS_BF16, "bad qtype");
        const int64_t n = s->n;
        const int64_t ldq = (n + 7) & ~(int64_t)7;
        const size_t esz = qtype == RGS_F64 ? 8 : (qtype == RGS_F32 ? 4 : 2);
        DevBuf Q, w, coef, part;
        Q.ensure(esz * (size_t)ldq * (ncols + 1));
        w.ensure(sizeof(double) * 2 * (size_t)n);
        coef.ensure(sizeof(double) * (size_t)ncols);
        part.ensure(sizeof(double) * 2 * (size_t)h->num_sms * kUpdMaxBlocksPerSm * s->k);
        // any finite data: the pass streams the same bytes whatever the values
        RGS_CUDA(cudaMemsetAsync(Q.ptr, 0, Q.bytes, h->stream));
        fill_kernel<<<h->num_sms * 4, 256, 0, h->stream>>>(w.as<double>(), 2 * n);
        RGS_CUDA(cudaGetLastError());
        RGS_CUDA(cudaMemsetAsync(coef.ptr, 0, coef.bytes, h->stream));
        const int saved = h->upd_blocks_per_sm;
        Events ev;
        float best = INFINITY;
        int best_c = saved;
        for (int c = 2; c <= kUpdMaxBlocksPerSm; ++c) {
            h->upd_blocks_per_sm = c;
            UpdateLaunch L{};
            L.n = n;
            L.ncols = ncols;
            L.Q = Q.ptr;
            L.ldq = ldq;
            L.qtype = qtype;
            L.w = w.as<double>();
            L.ldw = n;
            L.wcols = 1;
            L.coef = coef.as<double>();
            L.qout = Q.as<char>() + esz * (size_t)ncols * ldq;
            L.df_sketch = qtype != RGS_F64 ? 1 : 0;
            L.w_next = w.as<double>() + n;
            int np = 0;
            rgs_launch_update_sketch(h, s, L, part.as<double>(), &np, nullptr);     // warm-up
            RGS_CUDA(cudaEventRecord(ev.a, h->stream));
            for (int r = 0; r < 3; ++r) rgs_launch_update_sketch(h, s, L, part.as<double>(), &np, nullptr);
            RGS_CUDA(cudaEventRecord(ev.b, h->stream));
            RGS_CUDA(cudaEventSynchronize(ev.b));
            float t = 0.f;
            RGS_CUDA(cudaEventElapsedTime(&t, ev.a, ev.b));
            t /= 3.f;
            if (ms) ms[c - 2] = t;
            if (t < best) {
                best = t;
                best_c = c;
            }
        }
        h->upd_blocks_per_sm = best_c;
        if (out) fill_tuning(h, out);
    });
}

rgs_status rgs_autotune_batched(rgs_handle h, int32_t nbatch, const rgs_csr* A, const double* const* b,
                                const rgmres_batch_opts* opts, uint64_t sketch_seed, int32_t cycles,
                                rgs_tuning* out, float* ms) {
    if (!h) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_REQUIRE(nbatch >= 1 && A && b && opts, "empty batch");
        RGS_REQUIRE(cycles >= 1, "cycles must be >= 1");
        std::vector<rgmres_batch_opts> o(opts, opts + nbatch);
        size_t total = 0;
        for (auto& q : o) {
            q.max_cycles = cycles;
            q.fixed_steps = 1;
        }
        for (int i = 0; i < nbatch; ++i) total += (size_t)A[i].n;
        DevBuf xs;
        xs.ensure(sizeof(double) * total);
        std::vector<double*> xp(nbatch);
        size_t off = 0;
        for (int i = 0; i < nbatch; ++i) {
            xp[i] = xs.as<double>() + off;
            off += (size_t)A[i].n;
        }
        const int saved_b = h->batch_blocks_per_sm, saved_rr = h->batch_rr;
        const double saved_w = h->batch_min_team_work;
        const int rrs[2] = {4, 2};

        const double tw[3] = {131072.0, 524288.0, 2097152.0};
        Events ev;
        float best = INFINITY;
        int best_b = saved_b, best_rr = saved_rr;
        double best_w = saved_w;
        for (int ri = 0; ri < 2; ++ri) {
            // each compiled tile shape at its own occupancy limit and one below
            const int occ = rgs_batched_max_blocks_per_sm(opts[0].qtype, rrs[ri]);
            const int bpm[2] = {occ, std::max(1, occ - 1)};
            for (int bi = 0; bi < 2; ++bi)
            for (int wi = 0; wi < 3; ++wi) {
                const int c = (ri * 2 + bi) * 3 + wi;
                if (bi == 1 && !(bpm[1] < bpm[0])) {
                    if (ms) ms[c] = 0.f;
                    continue;
                }
                h->batch_rr = rrs[ri];
                h->batch_blocks_per_sm = bpm[bi];
                h->batch_min_team_work = tw[wi];
                RGS_CUDA(cudaMemsetAsync(xs.ptr, 0, xs.bytes, h->stream));
                RGS_CUDA(cudaEventRecord(ev.a, h->stream));
                const rgs_status st = rgmres_solve_batched(h, nbatch, A, b, xp.data(), o.data(), sketch_seed, nullptr);
                if (st != RGS_OK) {
                    h->batch_blocks_per_sm = saved_b;
                    h->batch_min_team_work = saved_w;
                    h->batch_rr = saved_rr;
                    throw RgsError{st, "batched solve failed while tuning: " + h->last_error};
                }
                RGS_CUDA(cudaEventRecord(ev.b, h->stream));
                RGS_CUDA(cudaEventSynchronize(ev.b));
                float t = 0.f;
                RGS_CUDA(cudaEventElapsedTime(&t, ev.a, ev.b));
                if (ms) ms[c] = t;
                if (t < best) {
                    best = t;
                    best_b = bpm[bi];
                    best_w = tw[wi];
                    best_rr = rrs[ri];
                }
            }
        }
        h->batch_blocks_per_sm = best_b;
        h->batch_min_team_work = best_w;
        h->batch_rr = best_rr;
        if (out) fill_tuning(h, out);
    });
}

}  // extern "C"
