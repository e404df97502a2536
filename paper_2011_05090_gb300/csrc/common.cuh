// Internal definitions shared by the librgs translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/librgs.h"

// ---------------------------------------------------------------- error plumbing
struct RgsError {
    rgs_status status;
    std::string msg;
};

#define RGS_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            throw RgsError{RGS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

#define RGS_REQUIRE(cond, what)                                                         \
    do {                                                                                \
        if (!(cond)) throw RgsError{RGS_ERR_INVALID_ARG, what};                         \
    } while (0)

// ---------------------------------------------------------------- device workspace
// A growable device buffer owned by a handle or an object.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    void ensure(size_t want) {
        if (want <= bytes) return;
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
        if (cudaMalloc(&ptr, want) != cudaSuccess) {
            cudaGetLastError();            // not sticky: keep it from surfacing at a later launch check
            ptr = nullptr;
            throw RgsError{RGS_ERR_ALLOC, "cudaMalloc of " + std::to_string(want) + " bytes failed"};
        }
        bytes = want;
    }
    template <typename T> T* as() const { return reinterpret_cast<T*>(ptr); }
    ~DevBuf() { if (ptr) cudaFree(ptr); }
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
};

// Device status words: [0] status code, [1] detail (column), [2..3] grid barrier count/generation.
struct rgs_context {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    std::string last_error;
    DevBuf ctl;            // int[kCtlWords]: status, detail, stop flag, barrier words (own lines), abort
    DevBuf trace;          // optional per-phase timestamps of the least-squares kernel
    DevBuf partials;       // per-CTA partial sketches
    DevBuf scratch;        // staging for host-pointer calls
    DevBuf lsbuf;          // Householder factors and vectors of the least-squares engine
    DevBuf work;           // P = Theta W, certificates
    DevBuf cert;           // rgs_certify_embedding: sketches, Gram matrices, Cholesky factor, Lanczos basis
    DevBuf cert_cols;      // rgs_certify_embedding: a chunk of V's columns in FP64
    int upd_blocks_per_sm = 4;             // tuning: CTAs per SM of the update / sketch pass (<= kUpdMaxBlocksPerSm)
    int ls_blocks = 0;     // cooperative grid of the least-squares kernel (at most num_sms)
    int ls_blocks_tuned = 0;   // tuning: 0 = one CTA per SM
    int precond_kind = 0;  // rgmres_set_preconditioner: RGS_PRECOND_*
    int precond_flexible = 0;
    void* precond_net = nullptr;           // RGS_PRECOND_LEARNED_CONV: the network
    const double* precond_field = nullptr; // and its second input channel (log kappa, H x W)
    rgs_callback_precond precond_cb{};     // RGS_PRECOND_CALLBACK: the caller's apply function
    DevBuf batch_theta;    // rgmres_solve_batched: shared BF16 Gaussian G (k x n)
    uint64_t batch_theta_seed = ~0ull;
    int batch_theta_k = 0;
    int64_t batch_theta_n = 0;
    int batch_blocks_per_sm = 0;           // tuning: 0 = the occupancy limit, at most 4
    int batch_rr = 4;                      // tuning: rows per thread of the batched kernel (2 or 4)
    double batch_min_team_work = 8192.0 * 64.0;   // tuning: rows x (k + restart) per CTA worth an extra CTA
    DevBuf batch_ws;       // per-instance workspaces of the batched solve
    DevBuf batch_desc;     // instance descriptors and team tables
    cudaStream_t capture_stream = nullptr; // private stream on which launches are captured into graphs
    cudaStream_t copy_stream = nullptr;    // host <-> device copies overlapped with rgs_qr
    int launches = 0;      // kernels launched by the current call
    int pdl = 1;           // launch the update and least-squares kernels with programmatic stream
                           // serialization (RGS_PDL=0 in the environment at rgs_create: plain order)
    int pdl_coop = 1;      // the driver accepts it together with a cooperative launch (cleared on refusal)
    std::vector<cudaEvent_t> events;   // pool for per-phase timings
    ~rgs_context() {
        for (auto e : events) cudaEventDestroy(e);
        if (capture_stream) cudaStreamDestroy(capture_stream);
        if (copy_stream) cudaStreamDestroy(copy_stream);
    }
};

// Accumulates the device time of repeated phases from pairs of events.
struct PhaseTimer {
    rgs_context* ctx;
    bool on;
    std::vector<std::pair<int, int>> marks[3];   // per phase: (start event, stop event)
    int next = 0;
    PhaseTimer(rgs_context* c, bool enabled) : ctx(c), on(enabled) {}
    int ev() {
        if (next >= (int)ctx->events.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) throw RgsError{RGS_ERR_CUDA, "cudaEventCreate failed"};
            ctx->events.push_back(e);
        }
        return next++;
    }
    int start(int phase) {
        if (!on) return -1;
        int a = ev();
        cudaEventRecord(ctx->events[a], ctx->stream);
        marks[phase].push_back({a, -1});
        return a;
    }
    void stop(int phase) {
        if (!on) return;
        int b = ev();
        cudaEventRecord(ctx->events[b], ctx->stream);
        marks[phase].back().second = b;
    }
    double total_ms(int phase) const {
        double t = 0.0;
        for (auto& m : marks[phase]) {
            float ms = 0.f;
            if (m.second >= 0 && cudaEventElapsedTime(&ms, ctx->events[m.first], ctx->events[m.second]) == cudaSuccess)
                t += ms;
        }
        return t;
    }
};

struct rgs_sketch_obj {
    rgs_handle h = nullptr;
    int kind = 0;
    int64_t n = 0, s = 0;
    int k = 0;
    uint64_t seed = 0;
    DevBuf theta;          // Gaussian: k x n FP64, column-major (ld k)
    DevBuf signbits;       // SRHT: ceil(n/32) words, bit set => -1
    DevBuf rows;           // SRHT: k int32 sample rows (ascending)
};

// Workspaces for partial sketches are sized for this many update CTAs per SM, whatever the
// tuning chooses at run time.
constexpr int kUpdMaxBlocksPerSm = 4;

// ---------------------------------------------------------------- device helpers
namespace rgsdev {

constexpr int kStatusWord = 0;
constexpr int kDetailWord = 1;
constexpr int kStopWord = 5;     // an Arnoldi cycle ended early (convergence or happy breakdown)
constexpr int kStepsWord = 6;    // Arnoldi steps of the cycle just solved
constexpr int kFlagWord = 7;     // set-up checks (e.g. a zero diagonal for Jacobi)
// the grid barrier's words sit on separate 128-byte lines so that polling one
// does not queue behind atomics on another
constexpr int kBarCount = 32;     // the barrier word
constexpr int kBarGen = 64;       // unused (kept free)
constexpr int kAbortWord = 96;
constexpr int kCtlWords = 128;   // words cleared at the start of every call
// After the cleared words: the clock-cycle budget of every device-side wait (int64; 0 = the
// default of 4e9 cycles, about two seconds), kept across calls (rgs_set_wait_budget).
constexpr int kBudgetWord = kCtlWords;
constexpr int kCtlAlloc = kCtlWords + 32;
constexpr long long kDefaultWaitCycles = 4000000000LL;

__device__ __forceinline__ long long wait_budget(const int* ctl) {
    const long long b = *reinterpret_cast<const volatile long long*>(ctl + kBudgetWord);
    return b > 0 ? b : kDefaultWaitCycles;
}

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 multiplies.
__host__ __device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = (uint32_t)p1;
        c[2] = n2;
        c[3] = (uint32_t)p0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__host__ __device__ inline double u53(uint32_t hi, uint32_t lo) {
    uint64_t v = (((uint64_t)hi << 32) | lo) >> 11;
    return ((double)v + 0.5) * 0x1p-53;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the block, valid in every thread, in a fixed order (deterministic).
// On this GPU a dependent FP64 add costs about 64 cycles, so the sum is a tree:
// a shuffle tree inside every warp, then one warp's tree over the warp totals.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sm /* >= NT/32 doubles */) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < NT / 32 ? sm[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) sm[NT / 32] = t;
    }
    __syncthreads();
    return sm[NT / 32];
}

// Double-float value hi + lo (two FP32 words, |lo| <= ulp(hi)/2): the compensated
// arithmetic used for the sketches of FP32 / BF16 bases.  Addition is Knuth's
// error-free TwoSum of the high words, the low words added to its error, and a
// final Dekker FastTwoSum renormalisation (about 2^-48 relative error per add).
struct df {
    float h, l;
};

__device__ __forceinline__ df df_add(df a, df b) {
    const float s = a.h + b.h;
    const float bv = s - a.h;
    float e = (a.h - (s - bv)) + (b.h - bv);
    e += a.l + b.l;
    const float h = s + e;
    return {h, e - (h - s)};
}
__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void red_add_release(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}


__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a cooperative launch on one word (the control word kBarCount, zero in
// its low 31 bits between barriers).  Every CTA arrives with a release reduction, whose reply
// nobody waits for: CTA 0 adds 2^31 - (G-1), the others 1, so the sum over one barrier is
// exactly 2^31 and the top bit flips when the last CTA arrives.  Thread 0 of each CTA reads the
// top bit once, before its first arrival (the bit cannot change before that arrival), and then
// polls with acquire loads for the alternating value.  Every wait is bounded: after the wait
// budget (by default 4e9 cycles, about two seconds) the waiting CTA records RGS_ERR_TIMEOUT,
// raises the abort word and returns false, and every other CTA then leaves at its next barrier.
struct GridBarrier {
    unsigned* word;
    unsigned expect;                       // thread 0: the top bit that completes the next barrier
    long long budget;                      // thread 0: clock cycles a wait may take
    unsigned raw_word;                     // thread 0: the two control words as read at construction,
    long long raw_budget;                  // turned into expect / budget at the first sync, so
    bool primed;                           // that the kernel's start does not wait for the reads
    __device__ explicit GridBarrier(int* ctl)
        : word(reinterpret_cast<unsigned*>(ctl + kBarCount)), expect(0u), budget(kDefaultWaitCycles), raw_word(0u),
          raw_budget(0), primed(false) {
        if (threadIdx.x == 0) {
            raw_word = ld_relaxed(word);
            raw_budget = *reinterpret_cast<const volatile long long*>(ctl + kBudgetWord);
        }
    }
    // ts (thread 0, optional): ts[0] = arrival of the whole CTA, ts[1] = departure (ns)
    __device__ bool sync(int* ctl, unsigned long long* ts = nullptr) {
        __shared__ int ok_sh;
        __syncthreads();                   // the CTA's writes are ordered before thread 0's release
        if (threadIdx.x == 0) {
            if (ts) ts[0] = globaltimer();
            if (!primed) {
                expect = (raw_word & 0x80000000u) ^ 0x80000000u;
                budget = raw_budget > 0 ? raw_budget : kDefaultWaitCycles;
                primed = true;
            }
            int ok = 1;
            red_add_release(word, blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u);
            const long long start = clock64();
            unsigned spins = 0;
            while ((ld_acquire(word) & 0x80000000u) != expect) {
                if (clock64() - start > budget) {
                    atomicCAS(ctl + kStatusWord, 0, (int)RGS_ERR_TIMEOUT);
                    atomicExch(ctl + kAbortWord, 1);
                    ok = 0;
                    break;
                }
                if ((++spins & 63u) == 0 && *reinterpret_cast<volatile int*>(ctl + kAbortWord) != 0) {
                    ok = 0;
                    break;
                }
            }
            expect ^= 0x80000000u;
            if (ts) ts[1] = globaltimer();
            ok_sh = ok;
        }
        __syncthreads();
        return ok_sh != 0;
    }
};

// Programmatic dependent launch: a kernel launched with programmatic stream serialization may
// start while the kernel before it on the stream is still running; pdl_wait() returns once that
// kernel has completed and its memory operations are visible (immediately for a plain launch).
// pdl_launch_dependents() lets the next such kernel be scheduled once every CTA of this grid has
// issued it (its CTAs then wait in their own pdl_wait()).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

}  // namespace rgsdev

// ---------------------------------------------------------------- launchers (host side)
// update.cu
struct UpdateLaunch {
    int64_t n;
    int ncols;              // prior basis columns used by the update
    const void* Q;          // basis (qtype), ld ldq
    int64_t ldq;
    int qtype;
    const double* w;        // input column(s), FP64, ld ldw between columns
    int64_t ldw;
    int wcols;              // number of input columns (batched sketches; no update when > 1)
    const double* wscale;   // optional device scalar multiplying w (FP64 w only)
    int w_df;               // w holds double-float pairs (float2) instead of FP64
    const double* coef;     // ncols FP64 coefficients (device)
    void* qout;             // optional stored result column (qtype)
    int df_sketch;          // SRHT transform sums: 0 FP64, 1 double-float (FP32 pairs), 2 FP32
    int no_gauss;           // Gaussian sketch with qout: store q'_i only (sketched later with another vector)
    int max_parts;          // 0, or an upper bound on the partial sketches per column
    const double* w_next;   // SRHT, wcols == 1: also sketch this FP64 column (no update) into the
                            // second block of partials (step 1 of the next column in the same pass)
};
// Number of partial sketches (per input column) the next update/sketch launch will write.
int rgs_update_nparts(const rgs_context* ctx, const rgs_sketch_obj* sk, int64_t n, int wcols);
// Largest gridDim.y of a launch: launches with one CTA row per column take at most this many.
constexpr int kMaxGridY = 65535;
// cudaPointerGetAttributes says host memory (or an address CUDA does not know).
bool rgs_is_host_pointer(const void* p);
// Y (k x ncols, ld ldy) = Theta X for FP64 device columns X (n x ncols, ld ldx), FP64 transform.
void rgs_sketch_columns(rgs_context* ctx, const rgs_sketch_obj* sk, int ncols, const double* X, int64_t ldx,
                        double* Y, int64_t ldy);
// Loads the no-allocation scratch array on `device` (current) and records its address.
void rgs_noalloc_reserve(int device);
int rgs_launch_update_sketch(rgs_context* ctx, const rgs_sketch_obj* sk, const UpdateLaunch& L,
                             double* partials, int* nparts, const int* ctl);
// Gaussian sketch partials of x1 (n entries, type x1type) and of the FP64 x2 in one pass over Theta;
// returns the partials per vector (the same count and values as two one-column launches).
int rgs_launch_gauss_sketch2(rgs_context* ctx, const rgs_sketch_obj* sk, int64_t n, const void* x1, int x1type,
                             const double* x2, double* part1, double* part2, const int* ctl);
void rgs_launch_reduce_partials(rgs_context* ctx, const double* partials, int nparts, int k, int ncols,
                                double scale, double* Y, int64_t ldy, bool df = false);
void rgs_launch_gaussian_theta(rgs_context* ctx, double* theta, int k, int64_t n, uint64_t seed);

// spmv.cu
// A sparse operator in SELL-32 form (sliced ELLPACK, Kreutzer et al. 2014, with slices of 32
// rows and no sorting): slice s holds rows 32 s .. 32 s + 31 padded to the slice's longest row,
// entry t of row 32 s + l at off[s] + 32 t + l (padding: value 0, column of a valid row).  A
// warp's load of entry t of its 32 rows is then one contiguous access.  Built once per solve.
struct SellView {
    int64_t nslices = 0;
    const int64_t* off = nullptr;   // nslices + 1 entry offsets
    const int32_t* col = nullptr;
    const void* val = nullptr;      // double-float pairs or FP64, 8 bytes an entry
};
struct SellBuf {
    DevBuf off, col, val;
    int64_t nslices = 0;
    int64_t entries = 0;
};
// The SELL-32 structure of A and its values (double-float pairs when dfm, else FP64) into sb;
// false (nothing built) when the padding would exceed a quarter of nnz.
bool rgs_build_sell(rgs_context* ctx, const rgs_csr& A, int dfm, SellBuf& sb);
// Values val (nnz, A's pattern) in sb's layout into out (sb.entries x 8 bytes).
void rgs_fill_sell_values(rgs_context* ctx, const rgs_csr& A, const double* val, int dfm, const SellBuf& sb,
                          DevBuf& out);
void rgs_csr_split_df(rgs_context* ctx, const double* val, int64_t nnz, void* out);
int rgs_spmv_nparts(const rgs_context* ctx, int64_t n, bool dfm);
// sell (optional, with an SRHT sketch): the product reads A in that layout instead of CSR (the
// same arithmetic in the same order: bit-identical results)
int rgs_launch_spmv(rgs_context* ctx, const rgs_csr& A, const void* vdf, const void* x, int xtype, void* w, int dfm,
                    const rgs_sketch_obj* sk, double* partials, const int* ctl, const double* yscale = nullptr,
                    const SellView* sell = nullptr);
int rgs_norm_grid(const rgs_context* ctx, int64_t n);
void rgs_launch_residual(rgs_context* ctx, const rgs_csr& A, const double* x, const double* b, double* r,
                         double* part, double* norm_out);
void rgs_launch_norm(rgs_context* ctx, int64_t n, const double* v, double* part, double* norm_out);
void rgs_launch_sol_update(rgs_context* ctx, int64_t n, const void* Q, int qtype, int64_t ldq, const double* cy,
                           double* x, const int* ctl, const double* rowscale = nullptr);
// x += z (z FP32 or FP64, n entries), skipped when the status word is set
void rgs_launch_add_vector(rgs_context* ctx, int64_t n, const void* z, int ztype, double* x, const int* ctl);
void rgs_launch_jacobi_setup(rgs_context* ctx, const rgs_csr& A, double* dinv, double* scaled_val);
// convnet.cu: z = M(x) = ||x|| net(x / ||x||, log kappa) for one grid vector x (xtype), z FP32
void rgs_convnet_apply_precond(rgs_context* ctx, void* net, const double* logkappa, const void* x, int xtype, float* z);
int64_t rgs_convnet_grid_points(const void* net);     // H x W of the network's grid
// batched.cu
int rgs_batched_max_blocks_per_sm(int qtype, int rr);
void rgs_launch_hess_solve(rgs_context* ctx, const double* Hr, int ldh, const double* g, const double* colscale,
                           int jmax, double* y, double* cy, int* ctl);
int rgs_multidot_grid(const rgs_context* ctx, int64_t n);
void rgs_launch_cgs_pass(rgs_context* ctx, int64_t n, const double* Vp, int64_t ldv, int ncols, const double* sigma,
                         double* w, double* part, double* coef, double* hacc, int accumulate, const int* ctl);
void rgs_launch_cgs_update(rgs_context* ctx, int64_t n, const double* Vp, int64_t ldv, int ncols, const double* coef,
                           double* w, double* out, double* part, const int* ctl);

// ls.cu: Householder (compact-WY) least-squares engine for the sketched problems.
struct LSState {
    int k, mmax;
    double *V, *VT, *T, *TT, *RinvT, *S;   // V column-major k x mmax; VT its row-major copy (ld mmax)
    double *sbuf, *pbuf, *ys, *yp;
    double *M;              // M = V T (column-major k x mmax): Q_H^T x = x - V (M^T x)
    double *u2s, *u2p;
    double *N;              // N = V T^T (column-major k x mmax): the new T column's sums over rows below i
    int* nfold;             // reflectors folded into N so far (phase 0 adds the newest once)
    double *d1, *d2;        // per-column dots (scratch)
    double *blk;            // 4 * grid
    double *sigma, *pnorm, *coef;
    double *R;
    int64_t ldr;
    double *cs, *sn, *g, *Hr;       // Givens state of the Hessenberg problem (GMRES); Hr ld mmax
    int max_parts;
    int fine_df;            // arithmetic of the internal arrays: 0 FP64, 1 double-float (FP32 / BF16 bases), 2 FP32
    int* ctl;
};
struct LSStep {
    int i;                  // reflectors already in the factorisation
    int append;             // append s_i (reduced from s_part) as column i
    int solve;              // solve for p and write x to R(:, xcol), coef
    int xcol;
    const double* s_part;
    int s_nparts;
    double s_scale;
    const double* p_vec;    // p given directly (scaled by p_scale), or
    const double* p_part;   // reduced from partials
    double* p_store;        // optional: the reduced p is also written here (FP64, k entries)
    int p_nparts;
    double p_scale;
    int p_lag;              // divide p by the r_ii of the appended column (Arnoldi lag)
    int s_df, p_df;         // partial sketches stored as double-float pairs (float2) instead of FP64
    int pnorm_idx;          // where to record ||p||
    unsigned long long* trace;  // optional: kLsTraceSlots timestamps (ns) per CTA, CTA b at trace + b * kLsTraceSlots
    int givens;             // GMRES: rotate H(:, i-1) = sigma_{i-1} R(0:i+1, i) once r_ii is known
    int arnoldi;            // a vanishing r_ii ends the cycle (happy breakdown) instead of failing
    double stop_tol;        // GMRES: stop the cycle when the rotated residual falls to this value
    int rich;               // step 2 by two Richardson sweeps on the normal equations (FP64 only)
};
void rgs_ls_alloc(DevBuf& buf, int k, int mmax, int grid, int max_parts, int fine_df, LSState* st);
void rgs_ls_reset(rgs_context* ctx, const LSState& st);
void rgs_launch_ls(rgs_context* ctx, const LSState& st, const LSStep& a);
int rgs_ls_max_blocks(int num_sms);
int rgs_ls_grid(const rgs_context* ctx);
// RGS_TRACE: summary of the least-squares timestamps of launches 0..m-1 on stderr
void rgs_print_ls_trace(rgs_context* h, int m, int grid);
// least-squares trace per CTA: start, (arrival, departure) at each of up to four grid barriers, end,
// end of phase 0's partial sums; inside the CTA's first phase-0 item: thread 0's sums done, shared
// sums visible, warp 0's totals done
constexpr int kLsTraceSlots = 14;
void rgs_launch_certificates(rgs_context* ctx, const double* S, int k, int m, const double* R, int64_t ldr,
                             const double* P, double* out2 /* device: delta, delta_tilde */, double* work);
