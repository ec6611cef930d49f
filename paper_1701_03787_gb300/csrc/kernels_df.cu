// Float-float sweeps: the paper's O(N) forward elimination and back substitution
// (Sec. 4: Helmholtz odd/even LU; Algorithm LUSolveBiharmonic with the Eq. ab tail)
// carried out in float-float arithmetic (value = hi + lo, two float32) with the float64
// LU factors stored as float-float pairs.
//
// GB300 runs float64 at about 1/64 of its float32 rate, while float-float keeps ~48
// significant bits on the float32 pipes.  The sweeps need no refinement step.
//
// Work decomposition: one thread per (mode, parity) chain, real and imaginary parts
// side by side.  The forward sweep writes y (float-float, 16 bytes per complex row) to
// the plan's spill scratch, [warp slot][row][lane], so a warp's 32 rows are one
// 512-byte line; the back substitution reads it back in reverse and writes u (float64),
// so u == f works.
#include <algorithm>

#include "chains.cuh"

namespace shen {
namespace {

using df::F2;

struct WorkItem {
    long col;
    int cls, par;
};

__device__ __forceinline__ bool work_item(const Plan &p, const int *order, long m0, long count, long tid,
                                          WorkItem &w) {
    if (tid >= 2 * count) return false;
    const long item = tid >> 1;
    w.par = (int)(tid & 1);
    const long mode = order ? (long)order[item] : m0 + item;
    w.col = mode - m0;
    w.cls = p.d_mode_class[mode];
    return true;
}

// Both kernels run a fixed grid of resident blocks.  Warp slot w (one per resident warp)
// takes the warp-sized groups of chains w, w + W, w + 2 W, ... (W slots) and spills its
// forward results to its own [row][lane] slice of the plan's scratch.
// Shape 1 is compiled for four blocks (16 warps) per SM, which lets it use 128 registers;
// left to itself the compiler picks 96 (five blocks).  Measured 6.67 against 6.91 ms at
// N = 1024, 1024 x 1024 (6.56 ms with its 5-row blocks); shape 0 would spill under that
// bound and keeps none.
template <int V>
__global__ void __launch_bounds__(128, V == 1 ? 4 : 0) helm_df_kernel(Plan p, const int *order, long m0, long count,
                                                      const double *f, double *u, float4 *scr) {
    const int lane = threadIdx.x & 31;
    const long slot = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
    const long nslots = ((long)gridDim.x * blockDim.x) >> 5;
    float4 *ys = scr + slot * (long)p.rows_h * 32 + lane;
    for (long t0 = slot * 32; t0 < 2 * count; t0 += nslots * 32) {
        WorkItem w;
        if (!work_item(p, order, m0, count, t0 + lane, w)) continue;
        const long off = 2 * w.col * (p.wall_first ? 1L : (long)p.N), rs = p.wall_first ? p.n_modes : 1L;
        const F2 h = df::from_f64((p.d_class_z2[w.cls] + p.c) * (kPi / 2));
        const long ch = 2L * w.cls + w.par, nch = 2 * p.n_classes;
        chains::solve_helm_df_chain<V>(p.N, w.par, f + off, u + off, chains::HelmDF{p.df_hb + ch, p.df_hf + ch, nch},
                                       h, ys, 32, rs);
    }
}

template <int V>
__global__ void __launch_bounds__(128) bih_df_kernel(Plan p, const int *order, long m0, long count,
                                                     const double *f, double *u, float4 *scr) {
    const int lane = threadIdx.x & 31;
    const long slot = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
    const long nslots = ((long)gridDim.x * blockDim.x) >> 5;
    float4 *ys = scr + slot * (long)p.rows_b * 32 + lane;
    for (long t0 = slot * 32; t0 < 2 * count; t0 += nslots * 32) {
        WorkItem w;
        if (!work_item(p, order, m0, count, t0 + lane, w)) continue;
        const long off = 2 * w.col * (p.wall_first ? 1L : (long)p.N), rs = p.wall_first ? p.n_modes : 1L;
        const long ch = 2L * w.cls + w.par, nch = 2 * p.n_classes;
        chains::solve_bih_df_chain<V>(p.N, w.par, f + off, u + off,
                                      chains::BihDF{p.df_bf + ch, p.df_bb0 + ch, p.df_bb1 + ch, p.df_bb2 + ch, nch},
                                      p.df_qs, ys, 32, rs);
    }
}

// Float32 sweeps over every mode (the solves inside shen_solve_refine): same
// decomposition and scratch as the float-float kernels.  ACC: u += H^-1 rhs.
template <bool ACC>
__global__ void __launch_bounds__(128) helm_f32_kernel(Plan p, const double *rhs, double *u, float4 *scr) {
    const int lane = threadIdx.x & 31;
    const long slot = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
    const long nslots = ((long)gridDim.x * blockDim.x) >> 5;
    float4 *ys = scr + slot * (long)p.rows_h * 32 + lane;
    for (long t0 = slot * 32; t0 < 2 * p.n_modes; t0 += nslots * 32) {
        WorkItem w;
        if (!work_item(p, p.d_order, 0, p.n_modes, t0 + lane, w)) continue;
        const long off = 2 * w.col * p.N;
        const float h = (float)((p.d_class_z2[w.cls] + p.c) * (kPi / 2));
        const long ch = 2L * w.cls + w.par, nch = 2 * p.n_classes;
        chains::solve_helm_f32_chain<ACC>(p.N, w.par, rhs + off, u + off,
                                          chains::HelmDF{p.df_hb + ch, p.df_hf + ch, nch}, h, ys, 32);
    }
}

template <bool ACC>
__global__ void __launch_bounds__(128) bih_f32_kernel(Plan p, const double *rhs, double *u, float4 *scr) {
    const int lane = threadIdx.x & 31;
    const long slot = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
    const long nslots = ((long)gridDim.x * blockDim.x) >> 5;
    float4 *ys = scr + slot * (long)p.rows_b * 32 + lane;
    for (long t0 = slot * 32; t0 < 2 * p.n_modes; t0 += nslots * 32) {
        WorkItem w;
        if (!work_item(p, p.d_order, 0, p.n_modes, t0 + lane, w)) continue;
        const long off = 2 * w.col * p.N;
        const long ch = 2L * w.cls + w.par, nch = 2 * p.n_classes;
        chains::solve_bih_f32_chain<ACC>(p.N, w.par, rhs + off, u + off,
                                         chains::BihDF{p.df_bf + ch, p.df_bb0 + ch, p.df_bb1 + ch, p.df_bb2 + ch, nch},
                                         p.df_qs, ys, 32);
    }
}

__device__ __forceinline__ float2 split2(double x) {
    const float hi = (float)x;
    return make_float2(hi, (float)(x - (double)hi));
}

// Float-float factor streams from the float64 factors, rows interleaved across chains:
// row i of chain ch = 2 class + parity goes to [i * nch + ch], nch = 2 n_classes.
__global__ void pack_helm_df_kernel(Plan p, float4 *hb, float2 *hf) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;      // chain-major row index
    const long nch = 2 * p.n_classes;
    if (t >= nch * p.rows_h) return;
    const long ch = t / p.rows_h, i = t % p.rows_h;
    const double *row = p.d_fac_h + t * kHelmF64;                    // 1/U0, U2, l
    const float2 a = split2(row[0]), b = split2(row[1]);
    hb[i * nch + ch] = make_float4(a.x, a.y, b.x, b.y);
    hf[i * nch + ch] = split2(row[2]);
}

__global__ void pack_bih_df_kernel(Plan p, float4 *bf, float4 *bb0, float4 *bb1, float2 *bb2) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const long nch = 2 * p.n_classes;
    if (t >= nch * p.rows_b) return;
    const long ch = t / p.rows_b, i = t % p.rows_b;
    const double *row = p.d_fac_b + t * kBiF64;                      // L1 L2 1/U0 U1 U2 ta tb
    float2 v[7];
    for (int q = 0; q < 7; q++) v[q] = split2(row[q]);
    const long o = i * nch + ch;
    bf[o] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    bb0[o] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
    bb1[o] = make_float4(v[4].x, v[4].y, v[5].x, v[5].y);
    bb2[o] = v[6];
}

__global__ void pack_qs_df_kernel(Plan p, float4 *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p.N + 8) return;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k < p.N - 4) {
        const float2 q = split2(p.tab.qk[k]), s = split2(p.tab.sk[k]);
        v = make_float4(q.x, q.y, s.x, s.y);
    }
    out[k] = v;
}

inline unsigned nblocks(long threads, int bs) { return (unsigned)((threads + bs - 1) / bs); }

}  // namespace

// Backing store: float4 streams first (16-byte aligned), then the float2 streams.
size_t df_table_floats(const Plan &p) {
    const size_t nch = 2 * (size_t)p.n_classes;
    return nch * ((size_t)p.rows_h * 4 + (size_t)p.rows_b * 12) + (size_t)(p.N + 8) * 4 +
           nch * ((size_t)p.rows_h * 2 + (size_t)p.rows_b * 2);
}

cudaError_t pack_df(Plan &p, cudaStream_t s) {
    const size_t nch = 2 * (size_t)p.n_classes;
    float4 *hb = reinterpret_cast<float4 *>(p.d_fac_df);
    float4 *bf = hb + nch * p.rows_h;
    float4 *bb0 = bf + nch * p.rows_b;
    float4 *bb1 = bb0 + nch * p.rows_b;
    float4 *qs = bb1 + nch * p.rows_b;
    float2 *hf = reinterpret_cast<float2 *>(qs + p.N + 8);
    float2 *bb2 = hf + nch * p.rows_h;
    p.df_hb = hb;
    p.df_hf = hf;
    p.df_bf = bf;
    p.df_bb0 = bb0;
    p.df_bb1 = bb1;
    p.df_bb2 = bb2;
    p.df_qs = qs;
    pack_helm_df_kernel<<<nblocks((long)nch * p.rows_h, 256), 256, 0, s>>>(p, hb, hf);
    pack_bih_df_kernel<<<nblocks((long)nch * p.rows_b, 256), 256, 0, s>>>(p, bf, bb0, bb1, bb2);
    pack_qs_df_kernel<<<nblocks(p.N + 8, 256), 256, 0, s>>>(p, qs);
    return cudaGetLastError();
}

cudaError_t launch_solve_df(const Plan &p, int problem, long m0, long count, const double *f, double *u,
                            cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    // wall-index-first fields: modes in their own order, so that a warp's rows are contiguous
    // (measured 14.3 / 10.0 ms at N = 1024, 1024 x 1024,
    // against 22.7 / 21.5 ms in the class order)
    const int *order = (m0 == 0 && count == p.n_modes && !p.wall_first) ? p.d_order : nullptr;
    const int pb = problem == SHEN_HELMHOLTZ ? 0 : 1;
    const int v = p.df_variant[pb];
    if (v >= 2 && !p.wall_first) return launch_solve_df2(p, problem, v == 2, m0, count, f, u, s);
    // never more blocks than the scratch has warp slots for (df_setup sized it for this grid)
    const unsigned g = (unsigned)std::min<long>(nblocks(2 * count, 128), p.df_grid[pb][v & 1]);
    if (problem == SHEN_HELMHOLTZ) {
        if (v != 1) helm_df_kernel<0><<<g, 128, 0, s>>>(p, order, m0, count, f, u, p.d_ys[0]);
        else helm_df_kernel<1><<<g, 128, 0, s>>>(p, order, m0, count, f, u, p.d_ys[0]);
    } else {
        if (v != 1) bih_df_kernel<0><<<g, 128, 0, s>>>(p, order, m0, count, f, u, p.d_ys[1]);
        else bih_df_kernel<1><<<g, 128, 0, s>>>(p, order, m0, count, f, u, p.d_ys[1]);
    }
    return cudaGetLastError();
}

cudaError_t launch_solve_f32(const Plan &p, int problem, bool acc, const double *rhs, double *u, cudaStream_t s) {
    if (p.n_modes <= 0) return cudaSuccess;
    const int pb = problem == SHEN_HELMHOLTZ ? 0 : 1;
    const unsigned g = (unsigned)std::max(1, p.f32_grid[pb]);
    if (problem == SHEN_HELMHOLTZ) {
        if (acc) helm_f32_kernel<true><<<g, 128, 0, s>>>(p, rhs, u, p.d_ys[0]);
        else helm_f32_kernel<false><<<g, 128, 0, s>>>(p, rhs, u, p.d_ys[0]);
    } else {
        if (acc) bih_f32_kernel<true><<<g, 128, 0, s>>>(p, rhs, u, p.d_ys[1]);
        else bih_f32_kernel<false><<<g, 128, 0, s>>>(p, rhs, u, p.d_ys[1]);
    }
    return cudaGetLastError();
}

cudaError_t df_setup(Plan &p, long long &bytes) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const void *kern[2][2] = {{(const void *)helm_df_kernel<0>, (const void *)helm_df_kernel<1>},
                                      {(const void *)bih_df_kernel<0>, (const void *)bih_df_kernel<1>}};
    // a launch covers at most all the plan's chains: no more blocks than that
    const int needed = (int)std::min<long>(nblocks(2 * p.n_modes, 128), 1L << 30);
    for (int pb = 0; pb < 2; pb++) {
        int most = 1;
        for (int v = 0; v < 2; v++) {
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern[pb][v], 128, 0);
            if (e != cudaSuccess) return e;
            p.df_grid[pb][v] = std::min(std::max(1, per_sm) * sms, needed);
            most = std::max(most, p.df_grid[pb][v]);
        }
        // float32 sweeps (shen_solve_refine): their own residency, within the scratch
        {
            const void *kf = pb == 0 ? (const void *)helm_f32_kernel<true> : (const void *)bih_f32_kernel<true>;
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, 128, 0);
            if (e != cudaSuccess) return e;
            p.f32_grid[pb] = std::max(1, std::min(std::min(std::max(1, per_sm) * sms, needed), most));
        }
        const size_t n = (size_t)most * 4 * (pb == 0 ? p.rows_h : p.rows_b) * 32;   // float4
        bytes += (long long)(n * sizeof(float4));
        e = cudaMalloc((void **)&p.d_ys[pb], n * sizeof(float4));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace shen
