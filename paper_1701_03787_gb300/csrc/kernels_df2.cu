// Float-float sweeps with the forward result kept on chip (row-block shape 2 of the
// single-plan float-float solves).
//
// The paper's O(N) sweeps (Sec. 4: the Helmholtz odd/even LU; Algorithm LUSolveBiharmonic
// with the tail of Eq. ab) run serially down each parity chain and back up, so the forward
// result y of every row must be kept until the back substitution reaches it: 8 bytes per
// row of each real chain in float-float.  The thread-per-chain kernels (shape 0 and 1) run
// 16 warps per SM, which puts ~600 MB of y in flight and sends it through DRAM (32 of
// their ~82 bytes per complex row).  Here:
//   - each lane runs ONE real chain (the real or the imaginary part of one parity chain of
//     one mode: lane = 4 j + 2 parity + part, 8 modes per warp), which halves the y each
//     lane holds while the four lanes of a mode still read and write whole 32-byte sectors;
//   - one CTA of 4 warps per SM (one warp per scheduler) keeps 128 chains in flight, and
//     their y lives in Tensor Memory (256 rows per lane) and shared memory (96 rows per
//     lane, beside the copy rings below) before any of it goes to a global spill: at
//     N = 1024 (510 rows per chain) 69 % of y stays on chip;
//   - each row's float-float sum is accumulated with one renormalisation (sweep2.cuh),
//     and f and the factor rows stream through per-lane cp.async rings in shared memory
//     (32 rows ahead in the forward sweep, 16 in the backward one), since 4 warps cannot
//     hide DRAM latency by occupancy.
// Same arithmetic as the other float-float shapes, same ordering of the terms within a
// row up to the accumulation (so results agree to rounding, not bit for bit).
#include <algorithm>

#include "chains.cuh"
#include "sweep2.cuh"

namespace shen {
namespace {

using df::F2;
using sw2::Acc;

constexpr int kRB = 4;                 // rows per block (both sweeps)
constexpr int kThreads = 128;          // 4 warps: one per SM sub-partition

// Where the forward result of block b lives: global spill [0, GB), shared memory
// [GB, GB + SB), Tensor Memory [GB + SB, nb).
struct Tiers {
    int nb, GB, SB, TB;
};

__device__ __forceinline__ Tiers tiers_of(int rows_max, int tmem_blocks, int smem_blocks) {
    Tiers t;
    t.nb = (rows_max + kRB - 1) / kRB;
    t.TB = min(t.nb, tmem_blocks);
    t.SB = min(t.nb - t.TB, smem_blocks);
    t.GB = t.nb - t.TB - t.SB;
    return t;
}

// This lane's chain in group g of 8 modes: lane = 4 j + 2 parity + part.
struct Lane {
    bool active;          // the lane's mode exists
    int par, ri;          // parity chain, real (0) / imaginary (1) part
    int rows;             // rows of the lane's chain
    int cls;
    long ch;              // chain index 2 class + parity
    long col;             // column of the mode relative to the field pointers
};

__device__ __forceinline__ Lane lane_of(const Plan &p, const int *order, long m0, long count, long g, int lane,
                                        int n) {
    Lane L;
    const long it = g * 8 + (lane >> 2);
    L.par = (lane >> 1) & 1;
    L.ri = lane & 1;
    L.active = it < count;
    const long mode = L.active ? (order ? (long)order[it] : m0 + it) : m0;
    L.col = mode - m0;
    L.cls = p.d_mode_class[mode];
    L.ch = 2L * L.cls + L.par;
    L.rows = (n - L.par + 1) / 2;
    return L;
}

// cp.async (global -> shared, bypassing registers), 16 bytes at a time through L2 only, so
// the streams do not evict the small per-N tables from L1; groups committed per block and
// waited for in order.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int D>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(D) : "memory");
}

// Per-warp streaming ring in shared memory: the rows of the next blocks of every lane's
// chain, copied ahead with cp.async, 16 bytes per row, lane and stream.  Forward slot: the
// complex element of f (the lane uses its part) and the forward factors; backward slot:
// the three backward factor rows and, for spilled blocks, y.  8-byte values are copied as
// the aligned 16-byte pair that holds them (the pair of parities of one class for the
// float2 factor streams, the pair of lanes 2j, 2j+1 for the spill).
constexpr int kDf = 8;                                    // forward slots: 32 rows in flight
constexpr int kDb = 4;                                    // backward slots: 16 rows in flight
constexpr int kFwdSlot = kRB * 32 * (16 + 16);           // 4 KB
constexpr int kBwdSlot = kRB * 32 * (16 + 16 + 16 + 16); // 8 KB
constexpr int kRingBytes = (kDf * kFwdSlot > kDb * kBwdSlot) ? kDf * kFwdSlot : kDb * kBwdSlot;   // per warp

// One launch covers modes [m0, m0 + count) (order: the plan's class order, full plan only).
// gsp: the per-warp global spill, GB blocks of [row][lane] float2 per warp slot.
// TM: keep the last tmem_blocks blocks of every chain in Tensor Memory (tcols columns per CTA).
// Shared memory: [16 B: TMEM address][rings: 4 x kRingBytes][y tier: smem_blocks x kRB x 128 float2].
template <int PB, bool TM>
__global__ void __launch_bounds__(kThreads, 1)
    df2_kernel(Plan p, const int *order, long m0, long count, const double *f, double *u, float2 *gsp,
               int tmem_blocks, int smem_blocks, int tcols) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *tm_slot = reinterpret_cast<uint32_t *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *ring = smem_raw + 16 + warp * kRingBytes;
    float2 *ysm = reinterpret_cast<float2 *>(smem_raw + 16 + (kThreads / 32) * kRingBytes);
    uint32_t tbase = 0;
    if (TM) {
        if (warp == 0) sw2::tmem_alloc(tm_slot, (uint32_t)tcols);
        sw2::tmem_fence_before();
        __syncthreads();
        sw2::tmem_fence_after();
        tbase = *tm_slot + ((uint32_t)(32 * warp) << 16);
    }
    const int N = p.N;
    const int n = PB == 0 ? N - 2 : N - 4;
    const int rows_max = (n + 1) / 2;
    const Tiers T = tiers_of(rows_max, TM ? tmem_blocks : 0, smem_blocks);
    const long slot = blockIdx.x * (long)(kThreads / 32) + warp;
    const long nslots = (long)gridDim.x * (kThreads / 32);
    float2 *gw = gsp + slot * (long)T.GB * kRB * 32;            // this warp's spill, [b][r][lane]
    const long nch = 2 * p.n_classes;
    const long ngroups = (count + 7) / 8;
    const F2 zero{0.f, 0.f};
    // ring views
    double2 *rf = reinterpret_cast<double2 *>(ring);                                // [kDf][kRB][32]
    float4 *rl = reinterpret_cast<float4 *>(ring + kDf * kRB * 32 * 16);           // [kDf][kRB][32]
    float4 *rb0 = reinterpret_cast<float4 *>(ring);                                 // [kDb][kRB][32]
    float4 *rb1 = rb0 + kDb * kRB * 32;
    float4 *rb2 = rb1 + kDb * kRB * 32;
    float4 *ryg = rb2 + kDb * kRB * 32;
    for (long g = slot; g < ngroups; g += nslots) {
        const Lane L = lane_of(p, order, m0, count, g, lane, n);
        const double *fp = f + 2 * L.col * (long)N + L.ri;        // part of element k at fp[2 k]
        double *up = u + 2 * L.col * (long)N + L.ri;
        F2 h = zero;                                               // Helmholtz: alpha pi / 2
        if (PB == 0) h = sw2::from_f64((p.d_class_z2[L.cls] + p.c) * (kPi / 2));

        // ---------------------------------------------------------------- forward sweep
        auto fissue = [&](int b) {
            if (b < T.nb) {
                const int s = b % kDf;
#pragma unroll
                for (int r = 0; r < kRB; r++) {
                    const int i = b * kRB + r;
                    const int e = (s * kRB + r) * 32 + lane;
                    if (L.active && i < L.rows) {
                        cp_async16(rf + e, fp - L.ri + 2 * (2L * i + L.par));
                        if (PB == 0) cp_async16(rl + e, p.df_hf + (((long)i * nch + L.ch) & ~1L));
                        else cp_async16(rl + e, p.df_bf + (long)i * nch + L.ch);
                    } else {
                        rf[e] = make_double2(0.0, 0.0);
                        rl[e] = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
            cp_async_commit();
        };
        F2 y1 = zero, y2 = zero;
#pragma unroll 1
        for (int b = 0; b < kDf - 1; b++) fissue(b);
#pragma unroll 1
        for (int b = 0; b < T.nb; b++) {
            fissue(b + kDf - 1);
            cp_async_wait<kDf - 1>();
            const int s = b % kDf;
            float yv[2 * kRB];
#pragma unroll
            for (int r = 0; r < kRB; r++) {
                const int e = (s * kRB + r) * 32 + lane;
                const float4 l = rl[e];
                const double2 fc = rf[e];
                Acc a = sw2::acc_start(sw2::from_f64(L.ri ? fc.y : fc.x));
                if (PB == 0) {
                    const bool odd = (L.ch & 1) != 0;          // the chain's half of the float2 pair
                    sw2::acc_sub_mul(a, odd ? F2{l.z, l.w} : F2{l.x, l.y}, y1);
                } else {
                    sw2::acc_sub_mul(a, F2{l.z, l.w}, y2);       // the y_{i-2} term first
                    sw2::acc_sub_mul(a, F2{l.x, l.y}, y1);
                }
                const F2 y = sw2::acc_done(a);
                y2 = y1;
                y1 = y;
                yv[2 * r] = y.hi;
                yv[2 * r + 1] = y.lo;
            }
            if (b < T.GB) {
#pragma unroll
                for (int r = 0; r < kRB; r++) gw[(b * kRB + r) * 32 + lane] = make_float2(yv[2 * r], yv[2 * r + 1]);
            } else if (b < T.GB + T.SB) {
#pragma unroll
                for (int r = 0; r < kRB; r++)
                    ysm[((b - T.GB) * kRB + r) * kThreads + threadIdx.x] = make_float2(yv[2 * r], yv[2 * r + 1]);
            } else if (TM) {
                __syncwarp();
                sw2::tmem_st8(tbase + 8u * (uint32_t)(b - T.GB - T.SB), yv);
            }
        }
        cp_async_wait<0>();
        if (TM) sw2::tmem_wait_st();

        // ---------------------------------------------------------------- back substitution
        // biharmonic: u_i = (y_i - ta Sq - tb Ss - U2 u_{i+2} - U1 u_{i+1}) / U0,
        //             Sq = sum_{j >= i+3} q_j u_j, Ss = sum_{j >= i+3} s_j u_j;
        // Helmholtz:  u_i = (y_i + h u_{i+1} - U2 S) / U0, S = sum_{j > i} u_j (kept in Sq).
        auto bissue = [&](int b) {
            if (b >= 0) {
                const int s = b % kDb;
#pragma unroll
                for (int r = 0; r < kRB; r++) {
                    const int i = b * kRB + r;
                    const int e = (s * kRB + r) * 32 + lane;
                    if (L.active && i < L.rows) {
                        const long o = (long)i * nch + L.ch;
                        if (PB == 0) {
                            cp_async16(rb0 + e, p.df_hb + o);
                        } else {
                            cp_async16(rb0 + e, p.df_bb0 + o);
                            cp_async16(rb1 + e, p.df_bb1 + o);
                            cp_async16(rb2 + e, p.df_bb2 + (o & ~1L));
                        }
                    } else {
                        rb0[e] = make_float4(0.f, 0.f, 0.f, 0.f);
                        rb1[e] = make_float4(0.f, 0.f, 0.f, 0.f);
                        rb2[e] = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    if (b < T.GB) cp_async16(ryg + e, gw + (b * kRB + r) * 32 + (lane & ~1));
                }
            }
            cp_async_commit();
        };
        F2 u1 = zero, u2 = zero, u3 = zero, Sq = zero, Ss = zero;
        auto yload = [&](uint32_t (&yt)[2 * kRB], int b) {
            if (TM && b >= 0 && b >= T.GB + T.SB) {
                __syncwarp();
                sw2::tmem_ld8(tbase + 8u * (uint32_t)(b - T.GB - T.SB), yt);
            }
        };
        auto brun = [&](uint32_t (&yt)[2 * kRB], int b) {
            if (b < 0) return;
            bissue(b - kDb + 1);
            cp_async_wait<kDb - 1>();
            const int s = b % kDb;
            float yv[2 * kRB];
            if (b < T.GB) {
#pragma unroll
                for (int r = 0; r < kRB; r++) {
                    const float4 v = ryg[(s * kRB + r) * 32 + lane];
                    yv[2 * r] = (lane & 1) ? v.z : v.x;
                    yv[2 * r + 1] = (lane & 1) ? v.w : v.y;
                }
            } else if (b < T.GB + T.SB) {
#pragma unroll
                for (int r = 0; r < kRB; r++) {
                    const float2 v = ysm[((b - T.GB) * kRB + r) * kThreads + threadIdx.x];
                    yv[2 * r] = v.x;
                    yv[2 * r + 1] = v.y;
                }
            } else if (TM) {
                __syncwarp();
                sw2::tmem_wait_ld(yt);
#pragma unroll
                for (int q = 0; q < 2 * kRB; q++) yv[q] = __uint_as_float(yt[q]);
            }
#pragma unroll
            for (int r = kRB - 1; r >= 0; r--) {
                const int i = b * kRB + r;
                const int e = (s * kRB + r) * 32 + lane;
                const bool ok = L.active && i < L.rows;
                const F2 yi{yv[2 * r], yv[2 * r + 1]};
                const float4 b0 = rb0[e];
                F2 ui;
                if (PB == 0) {
                    // u_i = inv0 (y_i - U2 S) + (inv0 h) u_{i+1}: only the last product waits for u_{i+1}
                    const F2 inv0{b0.x, b0.y}, U2{b0.z, b0.w};
                    Acc a = sw2::acc_start(yi);
                    sw2::acc_sub_mul(a, U2, Sq);
                    const F2 part = sw2::mul_n(inv0, sw2::acc_done(a));
                    const F2 w = sw2::mul_n(inv0, h);
                    ui = sw2::add_mul(part, w, u1);
                    if (!ok) ui = zero;
                    Sq = df::add(Sq, ui);
                } else {
                    {
                        // (q, s) of column k + 6 (in the table's range for every row: N + 8 entries)
                        const float4 qv = __ldg(p.df_qs + 2 * i + L.par + 6);
                        const F2 nq = sw2::add_mul(Sq, F2{qv.x, qv.y}, u3);
                        const F2 ns = sw2::add_mul(Ss, F2{qv.z, qv.w}, u3);
                        if (i + 3 < L.rows) {
                            Sq = nq;
                            Ss = ns;
                        }
                    }
                    const float4 b1 = rb1[e];
                    const float4 b2 = rb2[e];
                    const F2 inv0{b0.x, b0.y}, U1{b0.z, b0.w};
                    const F2 U2{b1.x, b1.y}, ta{b1.z, b1.w};
                    const F2 tb = (L.ch & 1) ? F2{b2.z, b2.w} : F2{b2.x, b2.y};
                    // u_i = inv0 (y_i - ta Sq - tb Ss - U2 u_{i+2}) - (inv0 U1) u_{i+1}: only the
                    // last product waits for u_{i+1}
                    Acc a = sw2::acc_start(yi);
                    sw2::acc_sub_mul(a, ta, Sq);
                    sw2::acc_sub_mul(a, tb, Ss);
                    sw2::acc_sub_mul(a, U2, u2);
                    const F2 part = sw2::mul_n(inv0, sw2::acc_done(a));
                    const F2 w = sw2::mul_n(inv0, U1);
                    Acc c = sw2::acc_start(part);
                    sw2::acc_sub_mul(c, w, u1);
                    ui = sw2::acc_done(c);
                    if (!ok) ui = zero;
                }
                if (ok) up[2 * (2L * i + L.par)] = sw2::to_f64(ui);
                u3 = u2;
                u2 = u1;
                u1 = ui;
            }
        };
#pragma unroll 1
        for (int j = 0; j < kDb - 1; j++) bissue(T.nb - 1 - j);
        {
            uint32_t ya[2 * kRB], yb[2 * kRB];
            yload(ya, T.nb - 1);
#pragma unroll 1
            for (int b = T.nb - 1; b >= 0; b -= 2) {
                yload(yb, b - 1);
                brun(ya, b);
                yload(ya, b - 2);
                brun(yb, b - 1);
            }
        }
        cp_async_wait<0>();
        // rows beyond the unknowns are written as 0
        if (L.active && L.par == 0)
            for (int k = n; k < N; k++) up[2L * k] = 0.0;
    }
    if (TM) {
        sw2::tmem_fence_before();
        __syncthreads();
        sw2::tmem_fence_after();
        if (warp == 0) sw2::tmem_dealloc(*tm_slot, (uint32_t)tcols);
    }
}

constexpr int kSmemLimit = 232448;                                  // 227 KB per block
constexpr int kSmemBlocks = (kSmemLimit - 16 - (kThreads / 32) * kRingBytes) / (kRB * kThreads * 8);   // 24
constexpr int kTmemCols = 512;

inline size_t smem_bytes(int blocks) {
    return 16 + (size_t)(kThreads / 32) * kRingBytes + (size_t)blocks * kRB * kThreads * 8;
}

template <int PB, bool TM>
const void *kern() {
    return (const void *)df2_kernel<PB, TM>;
}

}  // namespace

// Grid of the on-chip float-float sweeps: one CTA per SM, at most one warp slot per group of
// 8 modes.  Their global spill is allocated by df2_alloc, when a plan first selects shape 2
// or 3 (shen_plan_set_shape, shen_plan_autotune), so plans that never use them do not hold it.
cudaError_t df2_setup(Plan &p, long long &) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const void *ks[4] = {kern<0, false>(), kern<0, true>(), kern<1, false>(), kern<1, true>()};
    for (const void *k : ks) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(kSmemBlocks));
        if (e != cudaSuccess) return e;
    }
    const long groups = (p.n_modes + 7) / 8;
    p.df2_grid = (int)std::max(1L, std::min<long>(sms, (groups + 3) / 4));
    return cudaSuccess;
}

cudaError_t df2_alloc(Plan &p) {
    for (int pb = 0; pb < 2; pb++) {
        if (p.d_gsp[pb]) continue;
        const int n = pb == 0 ? p.N - 2 : p.N - 4;
        const int nb = ((n + 1) / 2 + kRB - 1) / kRB;
        const int GB = std::max(0, nb - kSmemBlocks);             // the larger spill: no Tensor Memory tier
        const size_t cnt = (size_t)p.df2_grid * (kThreads / 32) * GB * kRB * 32;
        if (cnt == 0) continue;
        const cudaError_t e = cudaMalloc((void **)&p.d_gsp[pb], cnt * sizeof(float2));
        if (e != cudaSuccess) return e;
        p.device_bytes += (long long)(cnt * sizeof(float2));
    }
    return cudaSuccess;
}

cudaError_t launch_solve_df2(const Plan &p, int problem, bool tmem, long m0, long count, const double *f,
                             double *u, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int *order = (m0 == 0 && count == p.n_modes) ? p.d_order : nullptr;
    const int pb = problem == SHEN_HELMHOLTZ ? 0 : 1;
    const long ngroups = (count + 7) / 8;
    const unsigned g = (unsigned)std::max(1L, std::min<long>(p.df2_grid, (ngroups + 3) / 4));
    const int tb = tmem ? kTmemCols / 8 : 0;
    const size_t sm = smem_bytes(kSmemBlocks);
    float2 *gsp = p.d_gsp[pb];
    if (pb == 0) {
        if (tmem) df2_kernel<0, true><<<g, kThreads, sm, s>>>(p, order, m0, count, f, u, gsp, tb, kSmemBlocks, kTmemCols);
        else df2_kernel<0, false><<<g, kThreads, sm, s>>>(p, order, m0, count, f, u, gsp, 0, kSmemBlocks, kTmemCols);
    } else {
        if (tmem) df2_kernel<1, true><<<g, kThreads, sm, s>>>(p, order, m0, count, f, u, gsp, tb, kSmemBlocks, kTmemCols);
        else df2_kernel<1, false><<<g, kThreads, sm, s>>>(p, order, m0, count, f, u, gsp, 0, kSmemBlocks, kTmemCols);
    }
    return cudaGetLastError();
}

}  // namespace shen

