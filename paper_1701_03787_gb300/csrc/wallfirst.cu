// Wall-normal transforms of fields stored wall-index-first (the paper's uhat(l, m, n)
// order, Sec. 2: element (m, k) at complex index k * n_modes + m).
//
// The transform kernels work on whole mode columns staged in shared memory by 1-D bulk
// copies, which needs each column contiguous.  A wall-first field is therefore brought to
// column order one chunk of modes at a time: a tiled transpose (32 x 32 complex values
// through shared memory, coalesced on both sides) gathers the chunk into the plan's
// staging buffer, the mode-major transform runs on it, and a second transpose scatters
// the result back.  The arithmetic is the mode-major transform's, so the result is the
// transpose of the mode-major result bit for bit.
#include <algorithm>

#include "shen_internal.h"

namespace shen {
namespace {

constexpr int kT = 32;   // transpose tile (complex values)

// dst[j * N + k] = src[k * rs + j] for j < cols, k < N  (rs: complex stride between rows k)
__global__ void __launch_bounds__(kT * 8) gather_kernel(const double2 *src, long rs, int N, long cols,
                                                        double2 *dst) {
    __shared__ double2 tile[kT][kT + 1];
    const long j0 = (long)blockIdx.x * kT;
    const int k0 = blockIdx.y * kT;
    for (int r = threadIdx.y; r < kT; r += blockDim.y) {
        const int k = k0 + r;
        const long j = j0 + threadIdx.x;
        if (k < N && j < cols) tile[r][threadIdx.x] = src[(long)k * rs + j];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < kT; r += blockDim.y) {
        const long j = j0 + r;
        const int k = k0 + threadIdx.x;
        if (k < N && j < cols) dst[j * N + k] = tile[threadIdx.x][r];
    }
}

// dst[k * rs + j] = src[j * N + k]
__global__ void __launch_bounds__(kT * 8) scatter_kernel(const double2 *src, int N, long cols, double2 *dst,
                                                         long rs) {
    __shared__ double2 tile[kT][kT + 1];
    const long j0 = (long)blockIdx.x * kT;
    const int k0 = blockIdx.y * kT;
    for (int r = threadIdx.y; r < kT; r += blockDim.y) {
        const long j = j0 + r;
        const int k = k0 + threadIdx.x;
        if (k < N && j < cols) tile[r][threadIdx.x] = src[j * N + k];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < kT; r += blockDim.y) {
        const int k = k0 + r;
        const long j = j0 + threadIdx.x;
        if (k < N && j < cols) dst[(long)k * rs + j] = tile[threadIdx.x][r];
    }
}

}  // namespace

long wall_first_chunk(const Plan &p) {
    // two staging buffers of 64 MB each (at least one mode)
    return std::max(1L, std::min<long>(p.n_modes, (64L << 20) / (16L * p.N)));
}

cudaError_t wall_first_setup(Plan &p, long long &bytes) {
    if (!p.wall_first) return cudaSuccess;
    const size_t n = (size_t)wall_first_chunk(p) * p.N * 2;          // two buffers of complex values
    bytes += (long long)(n * sizeof(double2));
    return cudaMalloc((void **)&p.d_wf_stage, n * sizeof(double2));
}

// Transform of the modes [0, count) of a wall-first field whose element (0, 0) is at
// in / out (row stride n_modes complex values), chunk by chunk through the staging buffers.
cudaError_t launch_transform_wall_first(const Plan &p, int kind, int space, long count, const double *in,
                                        double *out, cudaStream_t s) {
    const long C = wall_first_chunk(p);
    const int N = p.N;
    double2 *A = p.d_wf_stage, *Bs = p.d_wf_stage + (size_t)C * N;
    const dim3 block(kT, 8);
    for (long m = 0; m < count; m += C) {
        const long cols = std::min(C, count - m);
        const dim3 grid((unsigned)((cols + kT - 1) / kT), (unsigned)((N + kT - 1) / kT));
        gather_kernel<<<grid, block, 0, s>>>(reinterpret_cast<const double2 *>(in) + m, p.n_modes, N, cols, A);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = launch_transform(p, kind, space, cols, reinterpret_cast<const double *>(A),
                             reinterpret_cast<double *>(Bs), s);
        if (e != cudaSuccess) return e;
        scatter_kernel<<<grid, block, 0, s>>>(Bs, N, cols, reinterpret_cast<double2 *>(out) + m, p.n_modes);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace shen
