// Givens rotations for the Hessenberg least-squares problem of GMRES (Eq. hls), applied by
// one warp.  Applying the stored rotations G_0..G_{j-1} to a new column h is a first-order
// linear recurrence on the running entry ("carry"):
//     out_t = c_t carry_t + s_t h_{t+1},   carry_{t+1} = -s_t carry_t + c_t h_{t+1},
// i.e. carry_{t+1} = a_t carry_t + b_t with a_t = -s_t, b_t = c_t h_{t+1}.  The affine maps
// compose associatively, so the warp scans them (log2 32 levels) instead of walking j
// dependent FP64 steps, each of which costs tens of cycles on this GPU.
#pragma once

#include "common.cuh"

namespace rgsdev {

// Column j of H has entries hcol(0..j+1).  Rotates it by G_0..G_{j-1} (cs, sn), forms G_j,
// updates g (g[j], g[j+1]) and writes the rotated column to Hr(:, j) (ld ldh).  Returns
// |g[j+1]|, the residual norm of the least-squares problem after j+1 columns, in every lane.
// REG: for j <= 128, issue every load at once and keep the lane's rotations in registers (for
// callers with registers to spare; the same arithmetic either way).
template <bool REG = false, class HF>
__device__ double givens_column_warp(int j, HF hcol, double* cs, double* sn, double* g, double* Hr, int ldh) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int T = (j + 31) / 32;                 // rotations per lane
    const int t0 = lane * T, t1 = min(j, t0 + T);
    double gj = 0.0, h0 = 0.0;
    if (REG) {                                   // issued with the loads below, used at the end
        gj = g[j];
        h0 = hcol(0);
    }
    constexpr int TR = 4;                        // up to 4 rotations a lane (j <= 128): every load
    double cr[TR], sr[TR], hr[TR];               // issued at once and kept in registers
    if (REG && T <= TR) {
#pragma unroll
        for (int q = 0; q < TR; ++q) {
            const int t = t0 + q;
            const bool ok = t < t1;
            cr[q] = ok ? cs[t] : 1.0;
            sr[q] = ok ? sn[t] : 0.0;
            hr[q] = ok ? hcol(t + 1) : 0.0;
        }
    }
    double A = 1.0, B = 0.0;                     // composition of the lane's maps, in order
    if (REG && T <= TR) {
#pragma unroll
        for (int q = 0; q < TR; ++q)
            if (t0 + q < t1) {
                const double a = -sr[q], b = cr[q] * hr[q];
                B = fma(a, B, b);
                A = a * A;
            }
    } else {
        for (int t = t0; t < t1; ++t) {
            const double a = -sn[t], b = cs[t] * hcol(t + 1);
            B = fma(a, B, b);
            A = a * A;
        }
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {           // inclusive scan: lane L = M_L o ... o M_0
        const double Ap = __shfl_up_sync(FULL, A, o), Bp = __shfl_up_sync(FULL, B, o);
        if (lane >= o) {
            B = fma(A, Bp, B);
            A = A * Ap;
        }
    }
    double Ae = __shfl_up_sync(FULL, A, 1), Be = __shfl_up_sync(FULL, B, 1);
    if (lane == 0) { Ae = 1.0; Be = 0.0; }
    double carry = fma(Ae, REG ? h0 : hcol(0), Be);
    if (REG && T <= TR) {
#pragma unroll
        for (int q = 0; q < TR; ++q)
            if (t0 + q < t1) {
                Hr[(size_t)j * ldh + t0 + q] = fma(cr[q], carry, sr[q] * hr[q]);
                carry = fma(-sr[q], carry, cr[q] * hr[q]);
            }
    } else {
        for (int t = t0; t < t1; ++t) {
            const double h1 = hcol(t + 1);
            Hr[(size_t)j * ldh + t] = fma(cs[t], carry, sn[t] * h1);
            carry = fma(-sn[t], carry, cs[t] * h1);
        }
    }
    const double x = __shfl_sync(FULL, carry, 31);   // entry j after G_0..G_{j-1}
    const double y = hcol(j + 1);
    const double d = hypot(x, y);
    const double c = d == 0.0 ? 1.0 : x / d, s = d == 0.0 ? 0.0 : y / d;
    if (!REG) gj = g[j];
    __syncwarp();
    if (lane == 0) {
        cs[j] = c;
        sn[j] = s;
        Hr[(size_t)j * ldh + j] = d;
        g[j + 1] = -s * gj;
        g[j] = c * gj;
    }
    return fabs(s * gj);
}

}  // namespace rgsdev
