// Solves on HOST fields: the field is streamed through plan-owned device staging slots
// in chunks of whole modes.  For chunk c (slot c mod kSlots) the copy in, the solve (in
// place, on the device slot) and the copy out run on three internal streams ordered by
// events, so chunk c+1 is copied in while chunk c is solved and chunk c-1 copied out.
// A call starts after the work queued on the caller's stream and that stream waits for
// its last copy-out.  The internal streams and the chunk counter are the plan's, so
// calls made on two different caller streams queue behind each other chunk by chunk
// without the pipeline draining in between.
#include <algorithm>

#include "shen_internal.h"

namespace shen {

struct HostPipe {
    static constexpr int kSlots = 3;
    double *slot[kSlots] = {};
    long slot_modes = 0;                  // modes per chunk
    cudaStream_t in = nullptr, comp = nullptr, out = nullptr;
    cudaEvent_t loaded[kSlots] = {}, solved[kSlots] = {}, freed[kSlots] = {};
    cudaEvent_t start = nullptr, done_in = nullptr, done_comp = nullptr, done_out = nullptr;
    long chunk = 0;                       // chunks issued so far (slot = chunk % kSlots)
    bool ready = false;
    long long bytes = 0;
};

cudaError_t launch_solve_range(const Plan &p, int problem, int precision, long m0, long count, const double *f,
                               double *u, cudaStream_t s);   // plan.cu

namespace {

constexpr size_t kChunkBytes = (size_t)256 << 20;   // target size of one staging slot

cudaError_t pipe_init(const Plan &p, HostPipe &h) {
    h.slot_modes = std::max<long>(1, std::min<long>(p.n_modes, (long)(kChunkBytes / ((size_t)p.N * 16))));
    const size_t slot_bytes = (size_t)h.slot_modes * p.N * 16;
    for (int i = 0; i < HostPipe::kSlots; i++) {
        cudaError_t e = cudaMalloc((void **)&h.slot[i], slot_bytes);
        if (e != cudaSuccess) return e;
        h.bytes += (long long)slot_bytes;
        e = cudaEventCreateWithFlags(&h.loaded[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.solved[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.freed[i], cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaStreamCreateWithFlags(&h.in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h.comp, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h.out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.done_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.done_comp, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.done_out, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    h.ready = true;
    return cudaSuccess;
}

}  // namespace

void host_pipe_free(HostPipe *h) {
    if (!h) return;
    if (h->in) cudaStreamSynchronize(h->in);
    if (h->comp) cudaStreamSynchronize(h->comp);
    if (h->out) cudaStreamSynchronize(h->out);
    for (int i = 0; i < HostPipe::kSlots; i++) {
        cudaFree(h->slot[i]);
        if (h->loaded[i]) cudaEventDestroy(h->loaded[i]);
        if (h->solved[i]) cudaEventDestroy(h->solved[i]);
        if (h->freed[i]) cudaEventDestroy(h->freed[i]);
    }
    for (cudaEvent_t e : {h->start, h->done_in, h->done_comp, h->done_out})
        if (e) cudaEventDestroy(e);
    for (cudaStream_t s : {h->in, h->comp, h->out})
        if (s) cudaStreamDestroy(s);
    delete h;
}

long long host_pipe_bytes(const HostPipe *h) { return h ? h->bytes : 0; }

cudaError_t host_solve(Plan &p, HostPipe *&h, int problem, int precision, const double *f_host, double *u_host,
                       cudaStream_t user) {
    if (!h) {
        h = new (std::nothrow) HostPipe;
        if (!h) return cudaErrorMemoryAllocation;
    }
    if (!h->ready) {
        cudaError_t e = pipe_init(p, *h);
        if (e != cudaSuccess) {          // release what was made; the next call starts over
            host_pipe_free(h);
            h = nullptr;
            return e;
        }
    }
    // the pipeline starts after the work already on the caller's stream
    cudaError_t e = cudaEventRecord(h->start, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->in, h->start, 0);
    if (e != cudaSuccess) return e;
    const size_t row_bytes = (size_t)p.N * 16;
    for (long m0 = 0; m0 < p.n_modes; m0 += h->slot_modes) {
        const long count = std::min(h->slot_modes, p.n_modes - m0);
        const int s = (int)(h->chunk % HostPipe::kSlots);
        const size_t bytes = (size_t)count * row_bytes;
        const size_t off = (size_t)m0 * p.N * 2;      // doubles
        if (h->chunk >= HostPipe::kSlots) e = cudaStreamWaitEvent(h->in, h->freed[s], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->slot[s], f_host + off, bytes, cudaMemcpyHostToDevice, h->in);
        if (e == cudaSuccess) e = cudaEventRecord(h->loaded[s], h->in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->comp, h->loaded[s], 0);
        if (e == cudaSuccess) e = launch_solve_range(p, problem, precision, m0, count, h->slot[s], h->slot[s], h->comp);
        if (e == cudaSuccess) e = cudaEventRecord(h->solved[s], h->comp);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->out, h->solved[s], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(u_host + off, h->slot[s], bytes, cudaMemcpyDeviceToHost, h->out);
        if (e == cudaSuccess) e = cudaEventRecord(h->freed[s], h->out);
        if (e != cudaSuccess) return e;
        h->chunk++;
    }
    // the caller's stream continues once every copy out has landed
    e = cudaEventRecord(h->done_out, h->out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, h->done_out, 0);
    return e;
}

}  // namespace shen
