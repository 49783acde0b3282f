// Allocation-free variant of the policy-fixed multigrid solve for small
// Isaacs grids.  Some callers cannot let a library allocate device memory: a
// host that has handed every byte of the device to its own caching allocator,
// a real-time loop that must not pay for (or be stalled by) cudaMalloc /
// cudaFree and the device-wide synchronisation they can imply, or a code path
// that runs where CUDA allocation calls are not permitted.  This entry point
// takes all of its scratch from one file-scope device array instead; the
// caller passes the inputs and the output buffer.
#include <cstring>
#include <mutex>

#include "solver.cuh"

namespace gs {

namespace {

// Largest grid side served (2^7 - 1) and the scratch that covers it; every GPU
// that loads the library holds this array until the process exits.
constexpr int kStaticMaxSide = 127;
constexpr size_t kStaticBytes = (size_t)5 << 19;   // 2.5 MiB

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// Device address of g_static_scratch, looked up once per device with that
// device current (the host-side name is only a stand-in for the symbol).
constexpr int kMaxDevices = 64;
struct ScratchSlot {
    bool ready;
    unsigned char* ptr;
};
ScratchSlot g_slots[kMaxDevices];
std::mutex g_slots_mu;

unsigned char* scratch_base() {
    int dev = 0;
    GS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_last_error("static solve: device index %d out of range", dev);
        throw Error{GS_EINVAL};
    }
    std::lock_guard<std::mutex> lk(g_slots_mu);
    ScratchSlot& slot = g_slots[dev];
    if (!slot.ready) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_last_error("static solve: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            throw Error{GS_ECUDA};
        }
        slot.ptr = static_cast<unsigned char*>(p);
        slot.ready = true;
    }
    return slot.ptr;
}

// Bump carving of the scratch array (256-byte aligned pieces).
class Carver {
public:
    explicit Carver(unsigned char* base) : base_(base) {}
    template <typename T>
    T* take(size_t count) {
        const size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        if (off_ + bytes > kStaticBytes) {
            set_last_error("static solve: scratch of %zu bytes exceeded", kStaticBytes);
            throw Error{GS_ENOMEM};
        }
        T* p = reinterpret_cast<T*>(base_ + off_);
        off_ += bytes;
        return p;
    }

private:
    unsigned char* base_;
    size_t off_ = 0;
};

// Device memory of the current device, or managed memory.
bool is_device_pointer(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    if (at.type != cudaMemoryTypeDevice) return false;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.device == dev;
}

gs_status static_solve(int32_t side, int32_t variant, uint64_t seed, const double* xi,
                       const uint8_t* alpha, const uint8_t* beta, const double* w0, double* w,
                       int32_t precision, cudaStream_t st, gs_solve_stats* stats) {
    unsigned char* base = scratch_base();
    Carver cv(base);
    const size_t n = (size_t)side * side;
    const int m1 = variant == 1 ? 5 : 4;

    // a solver object that lives on the host stack and points into the scratch
    gs_solver s;
    gamesolve_default_options(&s.opt);
    s.opt.precision = precision;
    s.st = st;
    DevScalars host_sc{};
    MGState host_mg{};
    s.dsc = cv.take<DevScalars>(1);
    s.mgd = cv.take<MGState>(1);
    s.hsc = &host_sc;
    s.mgh = &host_mg;

    IsaacsGrid g;
    g.side = side;
    g.variant = variant;
    g.n = n;
    g.Kh = make_isaacs_consts(side, variant, s.opt.mu_mode);
    g.Kd = cv.take<IsaacsConsts>(1);
    g.r0 = cv.take<double>(n);
    g.v = w;                                   // the caller's output holds the iterate
    g.rhs = cv.take<double>(n);
    g.alpha = cv.take<uint8_t>(n);
    g.code = cv.take<uint8_t>(n);
    g.beta = cv.take<uint32_t>(n);
    g.beta4 = cv.take<uint8_t>(n);
    g.dstatus = cv.take<int>(4);
    uint8_t* beta_stage = cv.take<uint8_t>(n * m1);
    int* bad = cv.take<int>(2);
    int sd = side;
    while (true) {
        Level L;
        L.side = sd;
        L.n = (size_t)sd * sd;
        g.lv.push_back(L);
        if ((int)L.n <= s.opt.coarse_max || sd < 3) break;
        sd = (sd - 1) / 2;
    }
    for (size_t l = 0; l < g.lv.size(); ++l) {
        Level& L = g.lv[l];
        if (l > 0) {
            L.A64 = cv.take<double>(9 * L.n);
            L.A32 = cv.take<float>(9 * L.n);
            L.u64 = cv.take<double>(L.n);
            L.f64 = cv.take<double>(L.n);
        }
        L.r64 = cv.take<double>(L.n);
        L.u32 = cv.take<float>(L.n);
        L.f32 = cv.take<float>(L.n);
        L.r32 = cv.take<float>(L.n);
        if (l + 1 < g.lv.size()) {
            const size_t sc = (size_t)(L.side - 1) / 2;
            L.P64 = cv.take<double>(8 * (sc + 1) * (sc + 1));
            L.P32 = cv.take<float>(8 * (sc + 1) * (sc + 1));
        }
    }
    g.inv = cv.take<double>(g.lv.back().n * g.lv.back().n);

    // inputs -> scratch; what must start at zero is cleared here
    GS_CUDA(cudaMemcpyAsync(g.Kd, &g.Kh, sizeof(IsaacsConsts), cudaMemcpyHostToDevice, st));
    GS_CUDA(cudaMemsetAsync(g.dstatus, 0, 4 * sizeof(int), st));
    GS_CUDA(cudaMemsetAsync(bad, 0, 2 * sizeof(int), st));
    GS_CUDA(cudaMemsetAsync(g.beta4, 0, n, st));
    NoiseSrc ns{xi, seed, side, 1};
    launch_isaacs_r0(g.Kd, side, g.Kh.kappa, ns, g.r0, st);
    GS_CUDA(cudaMemcpyAsync(g.alpha, alpha, n, cudaMemcpyDeviceToDevice, st));
    GS_CUDA(cudaMemcpyAsync(beta_stage, beta, n * m1, cudaMemcpyDeviceToDevice, st));
    launch_check_actions(g.alpha, n, m1, bad, st);
    launch_check_actions(beta_stage, n * m1, 4, bad + 1, st);
    int hbad[2] = {0, 0};
    GS_CUDA(cudaMemcpyAsync(hbad, bad, sizeof hbad, cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    if (hbad[0] || hbad[1]) {
        set_last_error("static solve: action out of range");
        return GS_EINVAL;
    }
    launch_pack_beta(beta_stage, m1, n, g.beta, g.beta4, st);
    launch_isaacs_assemble(g.Kd, side, g.alpha, g.beta, g.r0, g.code, g.rhs, st);
    // w0 == w: the warm start is already in place
    if (w0 && w0 != w) GS_CUDA(cudaMemcpyAsync(w, w0, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    else if (!w0) GS_CUDA(cudaMemsetAsync(w, 0, n * sizeof(double), st));

    int cycles = 0;
    double res = 0.0;
    const bool exact = solve_policy_system(&s, g, &cycles, &res);
    GS_CUDA(cudaStreamSynchronize(st));
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        stats->cycles = cycles;
        stats->systems = 1;
        stats->levels = (int)g.lv.size();
        stats->res_inf = res;
        stats->converged = exact ? 1 : 0;
    }
    if (!exact) {
        set_last_error("static solve: %d cycles reached before the float64 floor", cycles);
        return GS_ENOTCONV;
    }
    return GS_OK;
}

}  // namespace

}  // namespace gs

using namespace gs;

extern "C" gs_status gamesolve_isaacs_policy_solve_static(int32_t side, int32_t variant,
                                                          uint64_t seed, const double* xi,
                                                          const uint8_t* alpha, const uint8_t* beta,
                                                          const double* w0, double* w,
                                                          int32_t precision, void* stream,
                                                          gs_solve_stats* stats) {
    if (side < 1 || ((side + 1) & side) != 0 || side > kStaticMaxSide) {
        set_last_error("static solve: side must be 2^k - 1 and at most %d", kStaticMaxSide);
        return GS_EINVAL;
    }
    if ((variant != 0 && variant != 1) || precision < GS_PREC_FP64 || precision > GS_PREC_MIXED_BF16 ||
        !alpha || !beta || !w) {
        set_last_error("static solve: invalid argument");
        return GS_EINVAL;
    }
    if (!is_device_pointer(alpha) || !is_device_pointer(beta) || !is_device_pointer(w) ||
        (w0 && !is_device_pointer(w0)) || (xi && !is_device_pointer(xi))) {
        set_last_error("static solve: every array must be device memory");
        return GS_EINVAL;
    }
    try {
        return static_solve(side, variant, seed, xi, alpha, beta, w0, w, precision,
                            (cudaStream_t)stream, stats);
    } catch (const Error& e) {
        return e.st;
    } catch (...) {
        set_last_error("static solve: unexpected host exception");
        return GS_ECUDA;
    }
}
