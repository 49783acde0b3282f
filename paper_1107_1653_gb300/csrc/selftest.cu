// Self-test of the bounded grid-wide barrier that every cooperative kernel of
// the library synchronises with.  One thread block of a cooperative launch
// stays away from the barrier, so the others' waits must give up after the
// limit, raise the barrier's error flag and return; the host reads the flag as
// GS_ETIMEOUT.  Nothing here traps or spins without a limit: the kernel ends
// on its own and the context stays usable.
#include <algorithm>

#include "gridsync.cuh"

namespace gs {

namespace {

constexpr int kSelfTestThreads = 128;

__global__ void __launch_bounds__(kSelfTestThreads) k_barrier_selftest(GridBarrier* bar, int absent,
                                                                       unsigned long long limit_ns,
                                                                       int rounds, int* passed) {
    GridSync G{bar, gridDim.x, limit_ns};
    if ((int)blockIdx.x == absent) return;   // this block never arrives
    for (int r = 0; r < rounds; ++r) {
        if (!G.sync()) return;
        if (threadIdx.x == 0) atomicAdd(passed, 1);
    }
}

struct SelfTestState {
    GridBarrier bar;
    int passed;
    int pad[3];
};

gs_status run_barrier_selftest(int blocks, int absent, uint64_t limit_ns, int rounds,
                               cudaStream_t st, int32_t* passed_out) {
    int dev = 0, sms = 0, per_sm = 0;
    GS_CUDA(cudaGetDevice(&dev));
    GS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_barrier_selftest,
                                                          kSelfTestThreads, 0));
    // a cooperative launch needs every block resident at once
    blocks = std::max(1, std::min(blocks, std::max(1, per_sm) * sms));
    SelfTestState* d = nullptr;
    GS_CUDA(cudaMallocAsync((void**)&d, sizeof(SelfTestState), st));
    SelfTestState h{};
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(SelfTestState), st);
    if (e == cudaSuccess) {
        GridBarrier* bar = &d->bar;
        int* passed = &d->passed;
        unsigned long long lim = limit_ns;
        void* args[] = {(void*)&bar, (void*)&absent, (void*)&lim, (void*)&rounds, (void*)&passed};
        e = cudaLaunchCooperativeKernel((const void*)k_barrier_selftest, dim3(blocks),
                                        dim3(kSelfTestThreads), args, 0, st);
        note_launches(1);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_last_error("barrier self-test: %s", cudaGetErrorString(e));
        return GS_ECUDA;
    }
    if (passed_out) *passed_out = h.passed;
    if (h.bar.error) {
        set_last_error("barrier self-test: a grid barrier wait gave up after %llu ns",
                       (unsigned long long)limit_ns);
        return GS_ETIMEOUT;
    }
    return GS_OK;
}

}  // namespace

}  // namespace gs

extern "C" gs_status gamesolve_selftest_barrier(int32_t blocks, int32_t absent_block,
                                                uint64_t limit_ns, int32_t rounds, void* stream,
                                                int32_t* passed) {
    if (blocks < 1 || rounds < 1 || rounds > 1000 || limit_ns < 1000 ||
        limit_ns > 100000000ull || absent_block >= blocks) {
        gs::set_last_error("barrier self-test: invalid argument");
        return GS_EINVAL;
    }
    try {
        return gs::run_barrier_selftest(blocks, absent_block, limit_ns, rounds,
                                        (cudaStream_t)stream, passed);
    } catch (const gs::Error& e) {
        return e.st;
    }
}
