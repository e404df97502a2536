// rgs_sketch_apply_noalloc: Y = Theta X without allocating any device memory during the call.
//
// rgs_sketch_apply keeps its per-CTA partial sketches in a workspace that the handle grows
// with cudaMalloc on demand.  Some callers cannot allow that: a cudaMalloc synchronises the
// device and can stall a latency-critical loop, and an application whose framework allocator
// already holds nearly all free device memory would see it fail.  This variant keeps the
// partial sketches in the fixed array below instead; everything else (kernels, sketch
// tables, the reduction into Y) is the same as in rgs_sketch_apply.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <string>

static constexpr size_t kScratchDoubles = RGS_NOALLOC_SCRATCH_BYTES / sizeof(double);

// Partial sketches of rgs_sketch_apply_noalloc (8 MiB on every device on which a handle is
// created, held until the process exits).  Shared by every call: calls whose work overlaps
// on the GPU (other streams, other host threads) race on it.  The kernels write every entry
// they later read, so nothing has to be cleared between calls.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

namespace {

// Host code may not use the array's name as a device address: its device address is looked
// up once per device, with that device current.  rgs_create does this for its device, so the
// module that holds the array is loaded (and the array reserved) when the handle is created,
// not during a later call; a call on a device without a handle would look it up itself.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

double* scratch_address(int device) {
    if (device < 0 || device >= kMaxDevices)
        throw RgsError{RGS_ERR_INVALID_ARG, "device ordinal beyond " + std::to_string(kMaxDevices)};
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_addr[device] == nullptr) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            throw RgsError{RGS_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array: ") +
                                             cudaGetErrorString(e)};
        g_addr[device] = static_cast<double*>(p);
    }
    return g_addr[device];
}

}  // namespace

void rgs_noalloc_reserve(int device) { (void)scratch_address(device); }

extern "C" rgs_status rgs_sketch_apply_noalloc(rgs_handle h, rgs_sketch s, int32_t ncols, const double* X,
                                               int64_t ldx, double* Y, int64_t ldy) {
    if (!h || !s) return RGS_ERR_INVALID_ARG;
    try {
        RGS_REQUIRE(ncols >= 0, "ncols must be >= 0");
        RGS_REQUIRE(ncols == 0 || (X && Y), "null X or Y");
        RGS_REQUIRE(ldx >= s->n && ldy >= s->k, "leading dimension too small");
        if (ncols == 0) return RGS_OK;
        const size_t per_part = (size_t)s->k * (size_t)ncols;       // one partial sketch for every column
        RGS_REQUIRE(per_part <= kScratchDoubles,
                    "k * ncols = " + std::to_string(per_part) + " exceeds the no-allocation scratch of " +
                        std::to_string(kScratchDoubles) + " doubles (RGS_NOALLOC_SCRATCH_BYTES); split the columns");
        RGS_REQUIRE(!rgs_is_host_pointer(X) && !rgs_is_host_pointer(Y), "X and Y must be device pointers");
        int device = -1;
        RGS_CUDA(cudaGetDevice(&device));
        RGS_REQUIRE(device == h->device, "the handle's device must be current");
        double* scratch = scratch_address(device);
        const double scale = s->kind == RGS_SKETCH_SRHT ? 1.0 / std::sqrt((double)s->k) : 1.0;
        // one CTA row per column: at most kMaxGridY columns per launch pair, in stream order
        for (int c0 = 0; c0 < ncols; c0 += kMaxGridY) {
            const int nc = std::min(ncols - c0, kMaxGridY);
            UpdateLaunch L{};
            L.n = s->n;
            L.ncols = 0;
            L.qtype = RGS_F64;
            L.w = X + (int64_t)c0 * ldx;
            L.ldw = ldx;
            L.wcols = nc;
            L.max_parts = (int)std::min<size_t>(kScratchDoubles / ((size_t)s->k * nc), 1u << 30);
            int nparts = 0;
            rgs_launch_update_sketch(h, s, L, scratch, &nparts, nullptr);
            rgs_launch_reduce_partials(h, scratch, nparts, s->k, nc, scale, Y + (int64_t)c0 * ldy, ldy);
        }
        h->last_error.clear();
        return RGS_OK;
    } catch (const RgsError& e) {
        h->last_error = e.msg;
        return e.status;
    } catch (const std::bad_alloc&) {
        h->last_error = "host allocation failed";
        return RGS_ERR_ALLOC;
    } catch (...) {
        h->last_error = "unexpected exception";
        return RGS_ERR_INVALID_ARG;
    }
}
