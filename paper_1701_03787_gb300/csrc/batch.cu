// Batched plans: many independent channels (instances) with uneven N, Fourier grids,
// nu and dt, solved in one persistent launch.
//
// Each instance is a channel as in shen_plan_create; its field is stored after the
// previous instance's (complex offset = sum of n_modes_j N_j over earlier instances).
// Plan time groups each instance's modes by z2 and factorises every distinct (instance,
// z2) once in float64 (Sec. 4 algorithms, as for single plans).  The solve is a
// persistent kernel: warps take chunks of 16 modes (32 parity chains) from a work queue
// ordered by decreasing N (longest chains first, equal N within a chunk), until the
// queue is empty.  The queue counter lives in plan-owned device memory and is reset by
// an asynchronous memset before each launch.
#include <algorithm>
#include <cmath>
#include <map>
#include <new>
#include <numeric>
#include <vector>

#include "chains.cuh"

namespace shen {

struct BatchInst {
    int N, rows_h, rows_b, tab;     // tab: index of the per-N table set
    long n_modes, mode0, col0;      // first global mode, first complex element of the field
    double c;
};

struct BatchCls {
    double z2;
    int inst;
    long fh, fb;                    // offsets (in rows) of the chain pair in the factor arrays
};

struct BatchDev {
    int n_inst;
    long n_modes, n_cls;
    const BatchInst *inst;
    const int *mode_inst, *mode_cls, *work;
    const BatchCls *cls;
    const RowTables *tabs;
    const float4 *qs_df;            // per table set: N_max + 8 entries each
    int qs_stride;
    double *fac_h, *fac_b;          // float64 factors, kHelmF64 / kBiF64 doubles per row
    // float-float factor streams, one block of rows per chain (stride 1), indexed by the
    // chain-row offsets of the float64 factors: Helmholtz hb (1/U0, U2), hf l;
    // biharmonic bf (L1, L2), bb0 (1/U0, U1), bb1 (U2, ta), bb2 tb
    float4 *df_hb, *df_bf, *df_bb0, *df_bb1;
    float2 *df_hf, *df_bb2;
    int *queue;
    int *err;
    // complex-element offset subtracted from every column offset: 0 for whole batched
    // fields; the first column of the chunk for a staging slot of the host pipeline
    long col_shift;
    // float-float spill scratch per problem, [warp slot][row][lane] (ys_rows rows per
    // slot); null: spill through the output column instead
    float4 *ys[2];
    int ys_rows[2];
};

namespace {

__global__ void batch_factor_kernel(BatchDev b) {
    const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (tid >= 2 * b.n_cls) return;
    const long c = tid >> 1;
    const int par = (int)(tid & 1);
    const BatchCls cl = b.cls[c];
    const BatchInst in = b.inst[cl.inst];
    const RowTables &T = b.tabs[in.tab];
    double *Fh = b.fac_h + (cl.fh + (long)par * in.rows_h) * kHelmF64;
    double *Fb = b.fac_b + (cl.fb + (long)par * in.rows_b) * kBiF64;
    chains::factor_helm_chain(T, in.N, cl.z2, in.c, par, Fh, in.rows_h, b.err, c);
    chains::factor_bih_chain(T, in.N, cl.z2, in.c, par, Fb, in.rows_b, b.err, c);
    // float-float copies (hi, lo) of the same rows
    const long oh = cl.fh + (long)par * in.rows_h, ob = cl.fb + (long)par * in.rows_b;
    auto split = [](double x) {
        const float hi = (float)x;
        return make_float2(hi, (float)(x - (double)hi));
    };
    for (int i = 0; i < in.rows_h; i++) {
        const double *r = Fh + i * kHelmF64;
        const float2 a = split(r[0]), bb = split(r[1]);
        b.df_hb[oh + i] = make_float4(a.x, a.y, bb.x, bb.y);
        b.df_hf[oh + i] = split(r[2]);
    }
    for (int i = 0; i < in.rows_b; i++) {
        const double *r = Fb + i * kBiF64;
        float2 v[7];
        for (int q = 0; q < 7; q++) v[q] = split(r[q]);
        b.df_bf[ob + i] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
        b.df_bb0[ob + i] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
        b.df_bb1[ob + i] = make_float4(v[4].x, v[4].y, v[5].x, v[5].y);
        b.df_bb2[ob + i] = v[6];
    }
}

__global__ void batch_pack_qs_kernel(BatchDev b, int n_tabs, const int *tab_N) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tabs * b.qs_stride) return;
    const int tab = t / b.qs_stride, k = t % b.qs_stride;
    const int N = tab_N[tab];
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k < N - 4) {
        const double q = b.tabs[tab].qk[k], s = b.tabs[tab].sk[k];
        const float qh = (float)q, sh = (float)s;
        v = make_float4(qh, (float)(q - (double)qh), sh, (float)(s - (double)sh));
    }
    const_cast<float4 *>(b.qs_df)[t] = v;
}

// precision: 0 float64, 1 float-float.  problem: SHEN_HELMHOLTZ / SHEN_BIHARMONIC.
// V: row-block shape of the float-float chains (identical results).
template <int PREC, int PROBLEM, int V>
__global__ void __launch_bounds__(128) batch_solve_kernel(BatchDev b, const double *f, double *u) {
    const int lane = threadIdx.x & 31;
    const long slot = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
    float4 *const scr = b.ys[PROBLEM == SHEN_HELMHOLTZ ? 0 : 1];
    float4 *const ys_slot = (PREC == 1 && scr)
                                ? scr + slot * (long)b.ys_rows[PROBLEM == SHEN_HELMHOLTZ ? 0 : 1] * 32 + lane
                                : nullptr;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(b.queue, 16);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= b.n_modes) return;
        const long item = base + (lane >> 1);
        const int par = lane & 1;
        if (item < b.n_modes) {
            const int m = b.work[item];
            const BatchInst in = b.inst[b.mode_inst[m]];
            const BatchCls cl = b.cls[b.mode_cls[m]];
            const long off = 2 * (in.col0 - b.col_shift + (long)(m - in.mode0) * in.N);
            if (PROBLEM == SHEN_HELMHOLTZ) {
                if (PREC == 0) {
                    chains::solve_helm_fp64_chain(in.N, par, f + off, u + off,
                                                  b.fac_h + (cl.fh + (long)par * in.rows_h) * kHelmF64,
                                                  (cl.z2 + in.c) * kPi / 2);
                } else {
                    const long oh = cl.fh + (long)par * in.rows_h;
                    // shape 1 fetches 4 rows per prefetch block here (96 registers, five blocks
                    // per SM): 6.74 ms on the 4096-instance workload against 6.97 ms with the
                    // single-plan kernel's 5 (122 registers); same bits at every depth
                    chains::solve_helm_df_chain_t<V == 0 ? 8 : 4>(
                        in.N, par, f + off, u + off, chains::HelmDF{b.df_hb + oh, b.df_hf + oh, 1},
                        df::from_f64((cl.z2 + in.c) * (kPi / 2)),
                        ys_slot ? ys_slot : chains::column_spill(u + off, par), ys_slot ? 32 : 2, 1L);
                }
            } else {
                if (PREC == 0) {
                    chains::solve_bih_fp64_chain(in.N, par, f + off, u + off,
                                                 b.fac_b + (cl.fb + (long)par * in.rows_b) * kBiF64,
                                                 b.tabs[in.tab].qk, b.tabs[in.tab].sk);
                } else {
                    const long ob = cl.fb + (long)par * in.rows_b;
                    chains::solve_bih_df_chain<V>(in.N, par, f + off, u + off,
                                                  chains::BihDF{b.df_bf + ob, b.df_bb0 + ob, b.df_bb1 + ob,
                                                                b.df_bb2 + ob, 1},
                                                  b.qs_df + (size_t)in.tab * b.qs_stride,
                                                  ys_slot ? ys_slot : chains::column_spill(u + off, par),
                                                  ys_slot ? 32 : 2);
                }
            }
        }
    }
}

using BatchKernel = void (*)(BatchDev, const double *, double *);

BatchKernel batch_kernel(int prec, int problem, int v) {
    if (prec == 0) return problem == SHEN_HELMHOLTZ ? batch_solve_kernel<0, SHEN_HELMHOLTZ, 0>
                                                    : batch_solve_kernel<0, SHEN_BIHARMONIC, 0>;
    if (problem == SHEN_HELMHOLTZ) return v ? batch_solve_kernel<1, SHEN_HELMHOLTZ, 1>
                                            : batch_solve_kernel<1, SHEN_HELMHOLTZ, 0>;
    return v ? batch_solve_kernel<1, SHEN_BIHARMONIC, 1> : batch_solve_kernel<1, SHEN_BIHARMONIC, 0>;
}

}  // namespace

void build_row_tables(int N, std::vector<double> &h, std::vector<float> &h32, int &stride, bool gl);   // plan.cu

}  // namespace shen

using namespace shen;

namespace shen {
struct BatchHostPipe;
void batch_host_free(BatchHostPipe *h);
long long batch_host_bytes(const BatchHostPipe *h);
}  // namespace shen

struct shen_batch_s {
    BatchDev d{};
    std::vector<BatchInst> inst;
    std::vector<int> work;                       // the work order (host copy), for the host pipeline
    BatchHostPipe *host = nullptr;               // shen_batch_solve_host's staging, built at its first call
    std::vector<int> tab_N;
    // owned device allocations
    std::vector<void *> allocs;
    RowTables *d_tabs = nullptr;
    long long device_bytes = 0;
    int grid[2][2][2] = {};                      // persistent grid per [precision][problem][shape]
    int auto_prec[2] = {SHEN_DF, SHEN_DF};       // SHEN_AUTO per problem (autotuned)
    int df_variant[2] = {0, 0};                  // float-float shape per problem (autotuned)
    ~shen_batch_s() {
        batch_host_free(host);
        for (void *p : allocs) cudaFree(p);
    }
};

namespace {

template <class T>
cudaError_t balloc(shen_batch_s *b, T **ptr, size_t count) {
    b->device_bytes += (long long)(count * sizeof(T));
    cudaError_t e = cudaMalloc((void **)ptr, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) b->allocs.push_back(*ptr);
    return e;
}

shen_status cuda_status(cudaError_t e) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SHEN_ERR_ALLOC : SHEN_ERR_CUDA;
}

}  // namespace

extern "C" {

shen_status shen_batch_plan_create(shen_batch_t *out, int n_inst, const shen_instance_desc *descs, unsigned flags,
                                   void *stream) {
    if (!out) return SHEN_ERR_ARG;
    *out = nullptr;
    if ((flags & ~SHEN_PLAN_GL) != 0 || n_inst < 1 || !descs) return SHEN_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // validate and lay out the instances
    std::vector<BatchInst> inst((size_t)n_inst);
    std::map<int, int> tab_of_N;
    long mode0 = 0, col0 = 0;
    for (int i = 0; i < n_inst; i++) {
        const shen_instance_desc &d = descs[i];
        if (d.N < 8 || d.N > 8192 || d.Nx < 2 || d.Nz < 2 || (d.Nx & 1) || (d.Nz & 1)) return SHEN_ERR_ARG;
        if (!(d.nu > 0) || !(d.dt > 0) || !(d.Lx > 0) || !(d.Lz > 0) || !std::isfinite(d.nu) ||
            !std::isfinite(d.dt) || !std::isfinite(d.Lx) || !std::isfinite(d.Lz))
            return SHEN_ERR_ARG;
        const double c = 2.0 / (d.nu * d.dt);
        if (!std::isfinite(c)) return SHEN_ERR_ARG;
        BatchInst &b = inst[i];
        b.N = d.N;
        b.rows_h = (d.N - 2 + 1) / 2;
        b.rows_b = (d.N - 4 + 1) / 2;
        b.n_modes = (long)(d.Nx / 2 + 1) * d.Nz;
        b.mode0 = mode0;
        b.col0 = col0;
        b.c = c;
        if (!tab_of_N.count(d.N)) {
            const int t = (int)tab_of_N.size();
            tab_of_N[d.N] = t;
        }
        b.tab = tab_of_N[d.N];
        mode0 += b.n_modes;
        col0 += b.n_modes * d.N;
        if (mode0 > (1L << 30)) return SHEN_ERR_ARG;
    }
    const long n_modes = mode0;
    // classes (distinct z2 per instance), factor offsets, per-mode lookups
    std::vector<BatchCls> cls;
    std::vector<int> mode_inst((size_t)n_modes), mode_cls((size_t)n_modes);
    long fh = 0, fb = 0;
    for (int i = 0; i < n_inst; i++) {
        const shen_instance_desc &d = descs[i];
        BatchInst &b = inst[i];
        const long nxh = d.Nx / 2 + 1;
        std::vector<std::pair<double, long>> z((size_t)b.n_modes);
        for (long ix = 0; ix < nxh; ix++)
            for (long iz = 0; iz < d.Nz; iz++) {
                const long kzi = iz < d.Nz / 2 ? iz : iz - d.Nz;
                const double kx = 2 * kPi * (double)ix / d.Lx, kz = 2 * kPi * (double)kzi / d.Lz;
                z[ix * d.Nz + iz] = {kx * kx + kz * kz, ix * d.Nz + iz};
            }
        std::sort(z.begin(), z.end());
        std::vector<int> lc((size_t)b.n_modes);       // mode -> distinct-z2 group
        std::vector<double> lz;
        for (long w = 0; w < b.n_modes; w++) {
            if (w == 0 || z[w].first != z[w - 1].first) lz.push_back(z[w].first);
            lc[z[w].second] = (int)lz.size() - 1;
        }
        // classes numbered by first appearance in mode order (nearby modes, nearby factors)
        std::vector<int> ren(lz.size(), -1);
        int next = 0;
        for (long m = 0; m < b.n_modes; m++)
            if (ren[lc[m]] < 0) ren[lc[m]] = next++;
        std::vector<double> cz(lz.size());
        for (size_t c = 0; c < lz.size(); c++) cz[ren[c]] = lz[c];
        const long cbase = (long)cls.size();
        for (size_t c = 0; c < cz.size(); c++) {
            cls.push_back(BatchCls{cz[c], i, fh, fb});
            fh += 2L * b.rows_h;
            fb += 2L * b.rows_b;
        }
        for (long m = 0; m < b.n_modes; m++) {
            mode_inst[b.mode0 + m] = i;
            mode_cls[b.mode0 + m] = (int)(cbase + ren[lc[m]]);
        }
    }
    // work order: decreasing N, then instance, then class
    std::vector<int> work((size_t)n_modes);
    std::iota(work.begin(), work.end(), 0);
    std::stable_sort(work.begin(), work.end(), [&](int a, int b2) {
        const int Na = inst[mode_inst[a]].N, Nb = inst[mode_inst[b2]].N;
        if (Na != Nb) return Na > Nb;
        if (mode_cls[a] != mode_cls[b2]) return mode_cls[a] < mode_cls[b2];
        return a < b2;
    });

    shen_batch_s *b = new (std::nothrow) shen_batch_s;
    if (!b) return SHEN_ERR_ALLOC;
    auto fail = [&](shen_status st) {
        delete b;
        return st;
    };
#define B_TRY(expr)                                  \
    do {                                             \
        cudaError_t e_ = (expr);                     \
        if (e_ != cudaSuccess) return fail(cuda_status(e_)); \
    } while (0)
    b->inst = inst;
    b->work = work;
    const int n_tabs = (int)tab_of_N.size();
    b->tab_N.assign((size_t)n_tabs, 0);
    int N_max = 0;
    for (auto &kv : tab_of_N) {
        b->tab_N[kv.second] = kv.first;
        N_max = std::max(N_max, kv.first);
    }
    // per-N row tables
    std::vector<RowTables> tabs_h((size_t)n_tabs);
    for (int t = 0; t < n_tabs; t++) {
        std::vector<double> tab;
        std::vector<float> tab32;
        int stride = 0;
        build_row_tables(b->tab_N[t], tab, tab32, stride, (flags & SHEN_PLAN_GL) != 0);
        double *dt = nullptr;
        B_TRY(balloc(b, &dt, tab.size()));
        B_TRY(cudaMemcpyAsync(dt, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        RowTables &T = tabs_h[t];
        T.bd0 = dt + 0 * stride; T.ad0 = dt + 1 * stride; T.adt = dt + 2 * stride;
        T.bb0 = dt + 3 * stride; T.bb2 = dt + 4 * stride; T.bb4 = dt + 5 * stride;
        T.ab0 = dt + 6 * stride; T.abp = dt + 7 * stride; T.abm = dt + 8 * stride;
        T.qb0 = dt + 9 * stride; T.pk = dt + 10 * stride; T.rk = dt + 11 * stride;
        T.qk = dt + 12 * stride; T.sk = dt + 13 * stride;
        T.qk32 = nullptr; T.sk32 = nullptr;
    }
    BatchDev &D = b->d;
    D.n_inst = n_inst;
    D.n_modes = n_modes;
    D.n_cls = (long)cls.size();
    D.qs_stride = N_max + 8;
    RowTables *d_tabs = nullptr;
    BatchInst *d_inst = nullptr;
    BatchCls *d_cls = nullptr;
    int *d_mi = nullptr, *d_mc = nullptr, *d_work = nullptr, *d_tabN = nullptr;
    float4 *d_qs = nullptr;
    B_TRY(balloc(b, &d_tabs, (size_t)n_tabs));
    B_TRY(balloc(b, &d_inst, inst.size()));
    B_TRY(balloc(b, &d_cls, cls.size()));
    B_TRY(balloc(b, &d_mi, (size_t)n_modes));
    B_TRY(balloc(b, &d_mc, (size_t)n_modes));
    B_TRY(balloc(b, &d_work, (size_t)n_modes));
    B_TRY(balloc(b, &d_tabN, (size_t)n_tabs));
    B_TRY(balloc(b, &d_qs, (size_t)n_tabs * D.qs_stride));
    B_TRY(balloc(b, &D.fac_h, (size_t)fh * kHelmF64));
    B_TRY(balloc(b, &D.fac_b, (size_t)fb * kBiF64));
    B_TRY(balloc(b, &D.df_hb, (size_t)fh));
    B_TRY(balloc(b, &D.df_hf, (size_t)fh));
    B_TRY(balloc(b, &D.df_bf, (size_t)fb));
    B_TRY(balloc(b, &D.df_bb0, (size_t)fb));
    B_TRY(balloc(b, &D.df_bb1, (size_t)fb));
    B_TRY(balloc(b, &D.df_bb2, (size_t)fb));
    B_TRY(balloc(b, &D.queue, 2));                   // one work-queue counter per problem
    B_TRY(balloc(b, &D.err, 4));
    B_TRY(cudaMemcpyAsync(d_tabs, tabs_h.data(), tabs_h.size() * sizeof(RowTables), cudaMemcpyHostToDevice, s));
    B_TRY(cudaMemcpyAsync(d_inst, inst.data(), inst.size() * sizeof(BatchInst), cudaMemcpyHostToDevice, s));
    B_TRY(cudaMemcpyAsync(d_cls, cls.data(), cls.size() * sizeof(BatchCls), cudaMemcpyHostToDevice, s));
    B_TRY(cudaMemcpyAsync(d_mi, mode_inst.data(), mode_inst.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    B_TRY(cudaMemcpyAsync(d_mc, mode_cls.data(), mode_cls.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    B_TRY(cudaMemcpyAsync(d_work, work.data(), work.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    B_TRY(cudaMemcpyAsync(d_tabN, b->tab_N.data(), b->tab_N.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    const int err_init[4] = {0, 0x7fffffff, 0, 0};
    B_TRY(cudaMemcpyAsync(D.err, err_init, sizeof(err_init), cudaMemcpyHostToDevice, s));
    D.inst = d_inst;
    D.cls = d_cls;
    D.mode_inst = d_mi;
    D.mode_cls = d_mc;
    D.work = d_work;
    D.tabs = d_tabs;
    D.qs_df = d_qs;
    b->d_tabs = d_tabs;
    batch_factor_kernel<<<(unsigned)((2 * D.n_cls + 127) / 128), 128, 0, s>>>(D);
    B_TRY(cudaGetLastError());
    batch_pack_qs_kernel<<<(unsigned)((n_tabs * D.qs_stride + 255) / 256), 256, 0, s>>>(D, n_tabs, d_tabN);
    B_TRY(cudaGetLastError());
    int err_host[2];
    B_TRY(cudaMemcpyAsync(err_host, D.err, sizeof(err_host), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaStreamSynchronize(s));
    if (err_host[0]) return fail(SHEN_ERR_SINGULAR);
    // persistent grids: the resident blocks of each solve kernel
    int dev = 0, sms = 0;
    B_TRY(cudaGetDevice(&dev));
    B_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    for (int pr = 0; pr < 2; pr++)
        for (int pb = 0; pb < 2; pb++)
            for (int v = 0; v < 2; v++) {
                int per_sm = 0;
                B_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel(pr, pb, v), 128, 0));
                b->grid[pr][pb][v] = std::max(1, sms * std::max(per_sm, 1));
            }
    // float-float spill scratch per problem: one [row][lane] slice per warp slot of the
    // larger float-float grid, rows of the largest instance
    int rows_max[2] = {1, 1};
    for (const BatchInst &in : inst) {
        rows_max[0] = std::max(rows_max[0], in.rows_h);
        rows_max[1] = std::max(rows_max[1], in.rows_b);
    }
    for (int pb = 0; pb < 2; pb++) {
        const long slots = 4L * std::max(b->grid[1][pb][0], b->grid[1][pb][1]);
        B_TRY(balloc(b, &b->d.ys[pb], (size_t)slots * rows_max[pb] * 32));
        b->d.ys_rows[pb] = rows_max[pb];
    }
#undef B_TRY
    *out = b;
    return SHEN_OK;
}

shen_status shen_batch_info(shen_batch_t batch, long *n_modes, long *field_elems, long *n_classes,
                            long long *device_bytes) {
    if (!batch) return SHEN_ERR_ARG;
    if (n_modes) *n_modes = batch->d.n_modes;
    if (field_elems) {
        const BatchInst &l = batch->inst.back();
        *field_elems = l.col0 + l.n_modes * l.N;
    }
    if (n_classes) *n_classes = batch->d.n_cls;
    if (device_bytes) *device_bytes = batch->device_bytes + batch_host_bytes(batch->host);
    return SHEN_OK;
}

shen_status shen_batch_offsets(shen_batch_t batch, long *offsets) {
    if (!batch || !offsets) return SHEN_ERR_ARG;
    for (size_t i = 0; i < batch->inst.size(); i++) offsets[i] = batch->inst[i].col0;
    const BatchInst &l = batch->inst.back();
    offsets[batch->inst.size()] = l.col0 + l.n_modes * l.N;
    return SHEN_OK;
}

namespace {
// One persistent launch of the solve kernel of (problem, precision) with the plan's
// float-float shape for that problem, on the grid sized for that kernel.
cudaError_t launch_batch(const shen_batch_s *batch, const BatchDev &D, int problem, int precision, const double *f,
                         double *u, cudaStream_t s) {
    const int pr = precision == SHEN_FP64 ? 0 : 1;
    const int pb = problem == SHEN_HELMHOLTZ ? 0 : 1;
    const int v = pr ? batch->df_variant[pb] : 0;
    batch_kernel(pr, problem, v)<<<batch->grid[pr][pb][v], 128, 0, s>>>(D, f, u);
    return cudaGetLastError();
}
}  // namespace

extern "C" shen_status shen_batch_solve(shen_batch_t batch, int problem, const double *f, double *u, int precision,
                                        void *stream) {
    if (!batch || !f || !u) return SHEN_ERR_ARG;
    if (problem != SHEN_HELMHOLTZ && problem != SHEN_BIHARMONIC) return SHEN_ERR_ARG;
    if (precision == SHEN_AUTO) precision = batch->auto_prec[problem];
    if (precision != SHEN_FP64 && precision != SHEN_DF) {
        if ((precision >= SHEN_FP32_R1 && precision <= SHEN_DF_R2) || precision == SHEN_FP64_R1)
            return SHEN_ERR_UNSUPPORTED;
        return SHEN_ERR_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(f) & 15u) || (reinterpret_cast<uintptr_t>(u) & 15u)) return SHEN_ERR_ARG;
    long elems = 0;
    shen_batch_info(batch, nullptr, &elems, nullptr, nullptr);
    if (f != u && !(f + 2 * elems <= u || u + 2 * elems <= f)) return SHEN_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    BatchDev D = batch->d;
    D.queue = batch->d.queue + problem;        // separate counters: a Helmholtz and a biharmonic
    cudaError_t e = cudaMemsetAsync(D.queue, 0, sizeof(int), s);   // solve may overlap
    if (e != cudaSuccess) return cuda_status(e);
    e = launch_batch(batch, D, problem, precision, f, u, s);
    return e == cudaSuccess ? SHEN_OK : cuda_status(e);
}

shen_status shen_batch_check(shen_batch_t batch) {
    if (!batch) return SHEN_ERR_ARG;
    int err_host[2];
    cudaError_t e = cudaMemcpy(err_host, batch->d.err, sizeof(err_host), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    return err_host[0] ? SHEN_ERR_SINGULAR : SHEN_OK;
}

shen_status shen_batch_autotune(shen_batch_t batch, int problem, const double *f, double *u, int *chosen, float *ms,
                                void *stream) {
    if (!batch || !f || !u) return SHEN_ERR_ARG;
    if (problem != SHEN_HELMHOLTZ && problem != SHEN_BIHARMONIC) return SHEN_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(f) & 15u) || (reinterpret_cast<uintptr_t>(u) & 15u)) return SHEN_ERR_ARG;
    long elems = 0;
    shen_batch_info(batch, nullptr, &elems, nullptr, nullptr);
    if (f == u || !(f + 2 * elems <= u || u + 2 * elems <= f)) return SHEN_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    BatchDev D = batch->d;
    D.queue = batch->d.queue + problem;
    const int pb = problem == SHEN_HELMHOLTZ ? 0 : 1;
    const int v0 = batch->df_variant[pb];
    const int cands[3][2] = {{SHEN_FP64, 0}, {SHEN_DF, 0}, {SHEN_DF, 1}};
    cudaEvent_t ev[2];
    if (cudaEventCreate(&ev[0]) != cudaSuccess) return cuda_status(cudaErrorUnknown);
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return cuda_status(cudaErrorUnknown);
    }
    float best = 0.f, best_df = 0.f;
    int pick = SHEN_DF, pick_df = v0;
    cudaError_t e = cudaSuccess;
    for (const auto &c : cands) {
        batch->df_variant[pb] = c[1];
        float t[3] = {0.f, 0.f, 0.f};
        for (int r = -1; r < 3 && e == cudaSuccess; r++) {     // r = -1: untimed
            e = cudaEventRecord(ev[0], s);
            if (e == cudaSuccess) e = cudaMemsetAsync(D.queue, 0, sizeof(int), s);
            if (e == cudaSuccess) e = launch_batch(batch, D, problem, c[0], f, u, s);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
            if (e == cudaSuccess && r >= 0) e = cudaEventElapsedTime(&t[r], ev[0], ev[1]);
        }
        if (e != cudaSuccess) break;
        std::sort(t, t + 3);
        if (best == 0.f || t[1] < best) {
            best = t[1];
            pick = c[0];
        }
        if (c[0] == SHEN_DF && (best_df == 0.f || t[1] < best_df)) {
            best_df = t[1];
            pick_df = c[1];
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e != cudaSuccess) {
        batch->df_variant[pb] = v0;
        return cuda_status(e);
    }
    batch->auto_prec[problem] = pick;
    batch->df_variant[pb] = pick_df;
    if (chosen) *chosen = pick;
    if (ms) *ms = best;
    return SHEN_OK;
}

void shen_batch_destroy(shen_batch_t batch) { delete batch; }

}  // extern "C"

// ---------------------------------------------------------------------------------
// Batched solves on HOST fields.  The batched field is cut into chunks of whole modes
// (contiguous in the field, at most kBatchChunkBytes each); chunk c goes through staging
// slot c mod 3: copy in, one persistent launch over the chunk's modes (its own work list,
// in the batch's decreasing-N order, and its own queue counter), copy out, on three
// internal streams ordered by events, so that copies in both directions overlap the
// solves of the neighbouring chunks.  Like shen_solve_host for single plans.
// ---------------------------------------------------------------------------------

namespace shen {

struct BatchHostPipe {
    static constexpr int kSlots = 3;
    double *slot[kSlots] = {};
    int *d_work = nullptr;                 // the chunks' work lists, one after the other
    int *d_queue = nullptr;                // queue counter of the pipeline's launches
    std::vector<long> m0, c0;              // chunk c: modes [m0[c], m0[c+1]), complex elements from c0[c]
    cudaStream_t in = nullptr, comp = nullptr, out = nullptr;
    cudaEvent_t loaded[kSlots] = {}, solved[kSlots] = {}, freed[kSlots] = {};
    cudaEvent_t start = nullptr, done_out = nullptr;
    long chunk = 0;                        // chunks issued so far (slot = chunk % kSlots)
    long long bytes = 0;
};

void batch_host_free(BatchHostPipe *h) {
    if (!h) return;
    for (cudaStream_t s : {h->in, h->comp, h->out})
        if (s) cudaStreamSynchronize(s);
    for (int i = 0; i < BatchHostPipe::kSlots; i++) {
        cudaFree(h->slot[i]);
        for (cudaEvent_t e : {h->loaded[i], h->solved[i], h->freed[i]})
            if (e) cudaEventDestroy(e);
    }
    cudaFree(h->d_work);
    cudaFree(h->d_queue);
    for (cudaEvent_t e : {h->start, h->done_out})
        if (e) cudaEventDestroy(e);
    for (cudaStream_t s : {h->in, h->comp, h->out})
        if (s) cudaStreamDestroy(s);
    delete h;
}

long long batch_host_bytes(const BatchHostPipe *h) { return h ? h->bytes : 0; }

namespace {

constexpr long kBatchChunkBytes = 256L << 20;   // target size of one staging slot

// Chunks, work lists and staging of a batched plan (blocking: the work lists are copied
// to the device synchronously).
cudaError_t batch_host_init(const shen_batch_s &b, BatchHostPipe &h) {
    const long cap = kBatchChunkBytes / 16;       // complex elements per slot (> 8192, the largest N)
    h.m0.assign(1, 0);
    h.c0.assign(1, 0);
    long used = 0, m = 0;
    for (const BatchInst &in : b.inst)
        for (long r = in.n_modes; r > 0;) {
            long fit = (cap - used) / in.N;
            if (fit == 0) {                       // close the chunk at mode m
                h.m0.push_back(m);
                h.c0.push_back(in.col0 + (m - in.mode0) * in.N);
                used = 0;
                fit = cap / in.N;
            }
            const long take = std::min(fit, r);
            used += take * in.N;
            m += take;
            r -= take;
        }
    const BatchInst &last = b.inst.back();
    h.m0.push_back(m);
    h.c0.push_back(last.col0 + last.n_modes * last.N);
    const long n_chunks = (long)h.m0.size() - 1;
    long span = 0;
    for (long c = 0; c < n_chunks; c++) span = std::max(span, h.c0[c + 1] - h.c0[c]);
    // each chunk's modes in the batch's work order (decreasing N, instance, class)
    std::vector<long> fill(h.m0.begin(), h.m0.end() - 1);
    std::vector<int> work((size_t)b.d.n_modes);
    for (int md : b.work) {
        const long c = (long)(std::upper_bound(h.m0.begin(), h.m0.end(), (long)md) - h.m0.begin()) - 1;
        work[(size_t)fill[c]++] = md;
    }
    cudaError_t e = cudaMalloc((void **)&h.d_work, work.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&h.d_queue, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(h.d_work, work.data(), work.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    h.bytes = (long long)(work.size() * sizeof(int) + sizeof(int));
    for (int i = 0; i < BatchHostPipe::kSlots; i++) {
        if ((e = cudaMalloc((void **)&h.slot[i], (size_t)span * 16)) != cudaSuccess) return e;
        h.bytes += (long long)span * 16;
        if ((e = cudaEventCreateWithFlags(&h.loaded[i], cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&h.solved[i], cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&h.freed[i], cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    for (cudaStream_t *s : {&h.in, &h.comp, &h.out})
        if ((e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&h.start, cudaEventDisableTiming)) != cudaSuccess) return e;
    return cudaEventCreateWithFlags(&h.done_out, cudaEventDisableTiming);
}

}  // namespace
}  // namespace shen

extern "C" shen_status shen_batch_solve_host(shen_batch_t batch, int problem, const double *f_host, double *u_host,
                                             int precision, void *stream) {
    if (!batch || !f_host || !u_host) return SHEN_ERR_ARG;
    if (problem != SHEN_HELMHOLTZ && problem != SHEN_BIHARMONIC) return SHEN_ERR_ARG;
    if (precision == SHEN_AUTO) precision = batch->auto_prec[problem];
    if (precision != SHEN_FP64 && precision != SHEN_DF) {
        if ((precision >= SHEN_FP32_R1 && precision <= SHEN_DF_R2) || precision == SHEN_FP64_R1)
            return SHEN_ERR_UNSUPPORTED;
        return SHEN_ERR_ARG;
    }
    long elems = 0;
    shen_batch_info(batch, nullptr, &elems, nullptr, nullptr);
    if (f_host != u_host && !(f_host + 2 * elems <= u_host || u_host + 2 * elems <= f_host)) return SHEN_ERR_ARG;
    if (!batch->host) {
        batch->host = new (std::nothrow) BatchHostPipe;
        if (!batch->host) return SHEN_ERR_ALLOC;
        const cudaError_t e = batch_host_init(*batch, *batch->host);
        if (e != cudaSuccess) {                   // release what was made; the next call starts over
            batch_host_free(batch->host);
            batch->host = nullptr;
            return cuda_status(e);
        }
    }
    BatchHostPipe &h = *batch->host;
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    // the pipeline starts after the work already on the caller's stream
    cudaError_t e = cudaEventRecord(h.start, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h.in, h.start, 0);
    const long n_chunks = (long)h.m0.size() - 1;
    for (long c = 0; c < n_chunks && e == cudaSuccess; c++) {
        const int s = (int)(h.chunk % BatchHostPipe::kSlots);
        const size_t bytes = (size_t)(h.c0[c + 1] - h.c0[c]) * 16;
        const size_t off = (size_t)h.c0[c] * 2;  // doubles
        BatchDev D = batch->d;
        D.work = h.d_work + h.m0[c];
        D.n_modes = h.m0[c + 1] - h.m0[c];
        D.col_shift = h.c0[c];
        D.queue = h.d_queue;
        if (h.chunk >= BatchHostPipe::kSlots) e = cudaStreamWaitEvent(h.in, h.freed[s], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.slot[s], f_host + off, bytes, cudaMemcpyHostToDevice, h.in);
        if (e == cudaSuccess) e = cudaEventRecord(h.loaded[s], h.in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h.comp, h.loaded[s], 0);
        if (e == cudaSuccess) e = cudaMemsetAsync(h.d_queue, 0, sizeof(int), h.comp);
        if (e == cudaSuccess) e = launch_batch(batch, D, problem, precision, h.slot[s], h.slot[s], h.comp);
        if (e == cudaSuccess) e = cudaEventRecord(h.solved[s], h.comp);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h.out, h.solved[s], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(u_host + off, h.slot[s], bytes, cudaMemcpyDeviceToHost, h.out);
        if (e == cudaSuccess) e = cudaEventRecord(h.freed[s], h.out);
        h.chunk++;
    }
    // the caller's stream continues once every copy out has landed
    if (e == cudaSuccess) e = cudaEventRecord(h.done_out, h.out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, h.done_out, 0);
    return e == cudaSuccess ? SHEN_OK : cuda_status(e);
}

// ---------------------------------------------------------------------------------
// No-allocation variant of the batched solve.
//
// Some callers cannot allocate device memory when they solve, for example an
// application whose device memory is divided up in advance by its own pool allocator,
// which must not see allocations it did not make during a time step.  For them,
// shen_batch_solve_noalloc keeps the only scratch
// the batched solve needs -- its work-queue counter -- in the fixed device array
// below instead of in memory owned by the plan.  The array is 256 bytes; every GPU
// that loads the library holds it until the process exits.
// ---------------------------------------------------------------------------------

namespace {

constexpr int kNoallocScratchWords = 64;                 // 256 bytes
static __device__ __align__(256) int g_noalloc_scratch[kNoallocScratchWords];   // [0]: queue counter

// Device address of g_noalloc_scratch in the current context, looked up on every call
// (cheap), so that a reset device or a new context never sees a stale address.
shen_status noalloc_scratch(int **out) {
    int *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&ptr), g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) return cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
    *out = ptr;
    return SHEN_OK;
}

}  // namespace

extern "C" shen_status shen_batch_solve_noalloc(shen_batch_t batch, int problem, const double *f, double *u,
                                                int precision, void *stream) {
    if (!batch || !f || !u) return SHEN_ERR_ARG;
    if (problem != SHEN_HELMHOLTZ && problem != SHEN_BIHARMONIC) return SHEN_ERR_ARG;
    if (precision == SHEN_AUTO) precision = batch->auto_prec[problem];
    if (precision != SHEN_FP64 && precision != SHEN_DF) {
        if ((precision >= SHEN_FP32_R1 && precision <= SHEN_DF_R2) || precision == SHEN_FP64_R1)
            return SHEN_ERR_UNSUPPORTED;
        return SHEN_ERR_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(f) & 15u) || (reinterpret_cast<uintptr_t>(u) & 15u)) return SHEN_ERR_ARG;
    long elems = 0;
    shen_batch_info(batch, nullptr, &elems, nullptr, nullptr);
    if (f != u && !(f + 2 * elems <= u || u + 2 * elems <= f)) return SHEN_ERR_ARG;
    int *scratch = nullptr;
    const shen_status st = noalloc_scratch(&scratch);
    if (st != SHEN_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the counter keeps the previous call's value: start it at zero
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_status(e);
    BatchDev D = batch->d;
    D.ys[0] = D.ys[1] = nullptr;              // spill through the output column: no plan scratch
    D.queue = scratch;
    e = launch_batch(batch, D, problem, precision, f, u, s);
    return e == cudaSuccess ? SHEN_OK : cuda_status(e);
}
