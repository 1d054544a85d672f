// C ABI of the cascaded central-moment step (declarations and documentation in include/cmlbm.h).
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/cmlbm.h"
#include "cm_launch.h"

#include <cstdlib>

// Device allocations that grow with the grid (state buffers, host staging, force field,
// turbulence scratch, the two-steps ring). Test hook: with CMLBM_TEST_ALLOC_LIMIT set to a
// byte count, any such allocation larger than it fails as if the device were out of memory, so
// that the CMLBM_ERR_NOMEM paths are tested without exhausting a shared GPU's memory.
static cudaError_t grid_alloc(void** p, size_t bytes) {
    if (const char* s = std::getenv("CMLBM_TEST_ALLOC_LIMIT")) {
        char* end = nullptr;
        const unsigned long long limit = std::strtoull(s, &end, 10);
        if (end != s && bytes > limit) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMalloc(p, bytes);
}

struct cmlbm {
    cmlbm_config cfg;
    cm::Params p;
    int D = 3;                 // 2 (D2Q9) or 3 (D3Q27)
    int Q = 27;
    size_t esize = 4;          // bytes per stored population
    size_t rsize = 4;          // bytes per arithmetic value (adjoint, force)
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;
    void* force = nullptr;     // [3][N] arithmetic type
    double* part = nullptr;    // reduction partials [kReduceMaxBlocks * 5]
    double* red = nullptr;     // reduction result [5]
    double* stage = nullptr;   // [4][N] FP64 staging for host buffers (allocated on first use)
    cudaStream_t st = nullptr;
    long long launches = 0;
    std::string err;
    // TMA-staged step: tensor maps of the two state buffers ({main, halo} each, 128 B apiece)
    bool tma = false;
    alignas(128) unsigned char maps[2][2][128];
    int* flag = nullptr;       // device error flag of the bounded pipeline waits
    // page-locked mirror of `flag` on TMA handles: refreshed by an asynchronous 4-byte copy after
    // every batch of TMA-staged steps, read by the host at the start of each call that returns
    // results and after each synchronising call, so that no call blocks just to check it
    volatile int* hflag = nullptr;
    int nsm = 0;
    void* turb = nullptr;      // [10][N] arithmetic type: rho, u, eddy stress (turbulence forcing)
    size_t ghost = 0;          // elements before the first own plane of a state buffer (nx ny on a slab)
    // CUDA graphs of two consecutive steps (state in buf[k] -> buf[1-k] -> buf[k]), one per
    // starting buffer, captured on a private stream and replayed on `st` by cmlbm_step; dropped
    // whenever the parameters or the force buffer change
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    // two steps per pass: the plane ring of the intermediate state (allocated on first use)
    bool two_steps = false;
    void* ring = nullptr;
    int pass_launches = 0;     // kernel launches of one two-step pass
#ifdef CM_NO_GRAPHS
    bool graphs = false;       // build option: plain launches only
#else
    bool graphs = true;        // false after a capture failed: plain launches from then on
#endif
    // split steps (cmlbm_step_split): the interior planes run on a private stream; ev_begin marks
    // the work issued on `st` before a split step, ev_interior the end of its interior launch
    cudaStream_t inner = nullptr;
    cudaEvent_t ev_begin = nullptr, ev_interior = nullptr;
    bool interior_pending = false;
    bool boundary_done = false;    // the boundary part of a split step was issued, its interior not yet
};

namespace {

thread_local std::string g_create_error;

int fail(cmlbm* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(cmlbm* h, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(h, CMLBM_ERR_CUDA, m);
}

// Test hook: with CMLBM_TEST_PIPELINE_FAULT set, every batch of TMA-staged steps is followed by
// a write of 1 into the handle's pipeline flag, the value a step kernel stores when a bounded
// wait runs out, so that the reporting below is tested without making any kernel wait in vain.
bool test_pipeline_fault() { return std::getenv("CMLBM_TEST_PIPELINE_FAULT") != nullptr; }

// Enqueue the refresh of the host mirror of the pipeline flag after TMA-staged steps.
cudaError_t mirror_flag(cmlbm* h) {
    if (!h->tma) return cudaSuccess;
    if (test_pipeline_fault()) {
        cudaError_t e = cudaMemsetAsync(h->flag, 1, 1, h->st);
        if (e != cudaSuccess) return e;
    }
    return cudaMemcpyAsync((void*)h->hflag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->st);
}

// CMLBM_ERR_CUDA if a TMA-staged step that has completed gave up on a bounded pipeline wait (its
// output, and everything computed from it since, is invalid). The flag is then cleared: the
// stream is drained so that no mirror copy still in flight sets it again.
int check_flag(cmlbm* h) {
    if (!h->tma || !h->hflag || *h->hflag == 0) return CMLBM_OK;
    cudaStreamSynchronize(h->st);
    cudaMemset(h->flag, 0, sizeof(int));
    *h->hflag = 0;
    return fail(h, CMLBM_ERR_CUDA, "a TMA-staged step gave up on a bounded pipeline wait");
}

// Switches to the handle's device for the duration of a call and restores the caller's.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { prev = -1; }
        if (prev != dev) ok = (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard() {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

size_t storage_size(int s) {
    switch (s) {
        case CMLBM_F64: return 8;
        case CMLBM_F32: return 4;
        case CMLBM_BF16: return 2;
        case CMLBM_F16: return 2;
    }
    return 0;
}

// Dispatch on (lattice, storage) to a launcher template.
template <class Fn>
cudaError_t dispatch(const cmlbm* h, Fn&& fn) {
    if (h->D == 3) {
        switch (h->cfg.storage) {
            case CMLBM_F64: return fn(std::integral_constant<int, 3>{}, (double*)nullptr);
            case CMLBM_F32: return fn(std::integral_constant<int, 3>{}, (float*)nullptr);
            case CMLBM_BF16: return fn(std::integral_constant<int, 3>{}, (__nv_bfloat16*)nullptr);
            case CMLBM_F16: return fn(std::integral_constant<int, 3>{}, (__half*)nullptr);
        }
    } else {
        switch (h->cfg.storage) {
            case CMLBM_F64: return fn(std::integral_constant<int, 2>{}, (double*)nullptr);
            case CMLBM_F32: return fn(std::integral_constant<int, 2>{}, (float*)nullptr);
            case CMLBM_BF16: return fn(std::integral_constant<int, 2>{}, (__nv_bfloat16*)nullptr);
            case CMLBM_F16: return fn(std::integral_constant<int, 2>{}, (__half*)nullptr);
        }
    }
    return cudaErrorInvalidValue;
}

// TMA-staged step when the handle has maps for src (one of its buffers, or maps made here).
cudaError_t do_step_tma(cmlbm* h, const void* map_main, const void* map_halo, const void* src, void* dst) {
    switch (h->cfg.storage) {
        case CMLBM_F32: return cm::launch_step_tma<float>(map_main, map_halo, src, dst, h->force, h->p, h->flag, h->nsm, h->st);
        case CMLBM_BF16: return cm::launch_step_tma<__nv_bfloat16>(map_main, map_halo, src, dst, h->force, h->p, h->flag, h->nsm, h->st);
        case CMLBM_F16: return cm::launch_step_tma<__half>(map_main, map_halo, src, dst, h->force, h->p, h->flag, h->nsm, h->st);
    }
    return cudaErrorInvalidValue;
}

// the kernels address a state buffer from its first own plane (past the ghost plane of a slab)
const void* own(const cmlbm* h, const void* b) { return (const char*)b + h->ghost * h->esize; }
void* own(const cmlbm* h, void* b) { return (char*)b + h->ghost * h->esize; }

cudaError_t do_step(cmlbm* h, const void* src, void* dst) {
    ++h->launches;
    if (h->tma) {
        for (int k = 0; k < 2; ++k)
            if (src == h->buf[k]) return do_step_tma(h, h->maps[k][0], h->maps[k][1], src, dst);
        alignas(128) unsigned char m[2][128];
        if (cm::encode_tma_maps(src, h->p, h->cfg.storage, m[0], m[1])) return do_step_tma(h, m[0], m[1], src, dst);
    }
    return dispatch(h, [&](auto d, auto* s) {
        using S = std::remove_pointer_t<decltype(s)>;
        return cm::launch_step<decltype(d)::value, S>(own(h, src), own(h, dst), h->force, h->p, h->st);
    });
}

// One step of the planes z0 .. z0 + nzc - 1 only (the pull still reads the whole source buffer),
// launched on stream `on`.
cudaError_t do_step_planes(cmlbm* h, const void* src, void* dst, int z0, int nzc, cudaStream_t on) {
    ++h->launches;
    cm::Params q = h->p;
    q.z0 = z0;
    q.nzc = nzc;
    return dispatch(h, [&](auto d, auto* s) {
        using S = std::remove_pointer_t<decltype(s)>;
        return cm::launch_step<decltype(d)::value, S>(own(h, src), own(h, dst), h->force, q, on);
    });
}

// Order the handle's stream after the interior launch of the last split step, so that whatever
// is issued on it next sees the whole new state.
cudaError_t join_interior(cmlbm* h) {
    if (!h->interior_pending) return cudaSuccess;
    h->interior_pending = false;
    return cudaStreamWaitEvent(h->st, h->ev_interior, 0);
}

void drop_graphs(cmlbm* h) {
    for (int k = 0; k < 2; ++k) {
        if (h->gexec[k]) cudaGraphExecDestroy(h->gexec[k]);
        h->gexec[k] = nullptr;
    }
}

// Enqueue two steps from buf[k]: buf[k] -> buf[1-k] -> buf[k] as two single steps, or, on a
// two-steps handle, one pass buf[k] -> buf[1-k] through the plane ring (the state then ends in
// buf[1-k]).
cudaError_t enqueue_two_steps(cmlbm* h, int k) {
    if (h->two_steps) {
        const int n = cm::launch_two_steps_f32(h->buf[k], h->buf[1 - k], h->ring, h->force, h->p, h->st);
        if (n < 0) return cudaErrorInvalidValue;
        h->pass_launches = n;
        h->launches += n;
        return cudaSuccess;
    }
    cudaError_t e = do_step(h, h->buf[k], h->buf[1 - k]);
    if (e == cudaSuccess) e = do_step(h, h->buf[1 - k], h->buf[k]);
    return e;
}

// Capture the two steps from buf[k] into an executable graph. Any failure leaves no capture
// open and returns the error (the caller then launches plainly).
cudaError_t capture_two_steps(cmlbm* h, int k, cudaGraphExec_t* out) {
    if (!h->cap) {
        cudaError_t e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    cudaStream_t saved = h->st;
    const long long launches = h->launches;
    h->st = h->cap;
    cudaError_t e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
    cudaError_t e1 = cudaSuccess, e2 = cudaSuccess;
    if (e == cudaSuccess) e1 = enqueue_two_steps(h, k);
    cudaGraph_t graph = nullptr;
    cudaError_t ee = (e == cudaSuccess) ? cudaStreamEndCapture(h->cap, &graph) : e;
    h->st = saved;
    h->launches = launches;
    if (e1 == cudaSuccess) e1 = e2;
    if (e1 == cudaSuccess) e1 = ee;
    if (e1 == cudaSuccess) e1 = cudaGraphInstantiate(out, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    return e1;
}

cudaError_t do_moments(cmlbm* h, const void* src, double* rho, double* u, int z0 = 0, int nzc = -1) {
    ++h->launches;
    return dispatch(h, [&](auto d, auto* s) {
        using S = std::remove_pointer_t<decltype(s)>;
        return cm::launch_moments<decltype(d)::value, S>(own(h, src), h->force, h->p, rho, u, h->st, z0,
                                                         nzc < 0 ? h->p.nz : nzc);
    });
}

int ensure_stage(cmlbm* h) {
    if (h->stage) return CMLBM_OK;
    cudaError_t e = grid_alloc((void**)&h->stage, sizeof(double) * 4 * (size_t)h->p.N);
    if (e != cudaSuccess) {
        h->stage = nullptr;
        cudaGetLastError();
        return fail(h, CMLBM_ERR_NOMEM, "cudaMalloc of the host staging buffer failed");
    }
    return CMLBM_OK;
}

bool valid_omega(double w) { return w > 0.0 && w < 2.0; }

}  // namespace

extern "C" {

int cmlbm_config_default(cmlbm_config* c) {
    if (!c) return CMLBM_ERR_INVALID;
    std::memset(c, 0, sizeof(*c));
    c->lattice = CMLBM_D3Q27;
    c->nx = c->ny = c->nz = 32;
    c->storage = CMLBM_F32;
    c->tau = 0.8;
    c->omega_3 = 1.0;
    c->omega_4 = 1.0;
    c->rho0 = 1.0;
    return CMLBM_OK;
}

const char* cmlbm_last_error(const cmlbm_t* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int cmlbm_create(const cmlbm_config* cfg, cmlbm_t** out) {
    if (!out) return fail(nullptr, CMLBM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, CMLBM_ERR_INVALID, "cfg is NULL");
    const cmlbm_config& c = *cfg;
    if (c.lattice != CMLBM_D2Q9 && c.lattice != CMLBM_D3Q27) return fail(nullptr, CMLBM_ERR_INVALID, "unknown lattice");
    if (storage_size(c.storage) == 0) return fail(nullptr, CMLBM_ERR_INVALID, "unknown storage");
    if (c.nx < 1 || c.ny < 1 || c.nz < 1) return fail(nullptr, CMLBM_ERR_INVALID, "grid sizes must be >= 1");
    if (c.lattice == CMLBM_D2Q9 && c.nz != 1) return fail(nullptr, CMLBM_ERR_INVALID, "D2Q9 needs nz == 1");
    const long long N = (long long)c.nx * c.ny * c.nz;
    if (N >= (1LL << 31)) return fail(nullptr, CMLBM_ERR_INVALID, "nx*ny*nz must be < 2^31");
    // D3Q27 grids with Q*N >= 2^32 elements run kernel variants with 64-bit element offsets
    const bool big = N * (c.lattice == CMLBM_D3Q27 ? 27 : 9) >= (1LL << 32);
    if (big && c.lattice != CMLBM_D3Q27)
        return fail(nullptr, CMLBM_ERR_INVALID, "D2Q9 grids need 9*nx*ny < 2^32 (32-bit element offsets)");
    if (c.nz > 65535) return fail(nullptr, CMLBM_ERR_INVALID, "nz must be <= 65535");
    if (c.ny > 65535) return fail(nullptr, CMLBM_ERR_INVALID, "ny must be <= 65535");
    for (int a = 0; a < 3; ++a)
        if (c.bc[a] != CMLBM_PERIODIC && c.bc[a] != CMLBM_BOUNCEBACK && !(a == 2 && c.bc[a] == CMLBM_HALO))
            return fail(nullptr, CMLBM_ERR_INVALID,
                        "bc must be CMLBM_PERIODIC or CMLBM_BOUNCEBACK (or CMLBM_HALO on z)");
    if (c.kernel < CMLBM_KERNEL_AUTO || c.kernel > CMLBM_KERNEL_PAIR_TWO_STEPS)
        return fail(nullptr, CMLBM_ERR_INVALID, "unknown kernel");
    const bool slab = c.bc[2] == CMLBM_HALO;
    if (slab && c.lattice != CMLBM_D3Q27) return fail(nullptr, CMLBM_ERR_INVALID, "CMLBM_HALO needs D3Q27");
    const long long S = slab ? (long long)c.nx * c.ny * (c.nz + 2) : N;
    if (slab && S * (c.lattice == CMLBM_D3Q27 ? 27 : 9) >= (1LL << 32))
        return fail(nullptr, CMLBM_ERR_INVALID, "Q*nx*ny*(nz+2) must be < 2^32 on a slab (32-bit element offsets)");
    if (big) {
        const bool pair_ok = c.storage != CMLBM_F64 && c.bc[0] == CMLBM_PERIODIC && c.nx % 64 == 0;
        if (c.storage != CMLBM_F64 && !pair_ok)
            return fail(nullptr, CMLBM_ERR_UNSUPPORTED,
                        "grids with 27*N >= 2^32 need FP64 storage, or periodic x and nx a multiple of 64 "
                        "(the two-cells-per-thread kernel)");
        if (c.kernel == CMLBM_KERNEL_TMA || c.kernel == CMLBM_KERNEL_PAIR_TWO_STEPS ||
            (c.kernel == CMLBM_KERNEL_DIRECT && c.storage != CMLBM_F64))
            return fail(nullptr, CMLBM_ERR_UNSUPPORTED,
                        "grids with 27*N >= 2^32 run the automatic kernel choice only (64-bit offsets)");
    }
    if (slab && c.kernel == CMLBM_KERNEL_TMA)
        return fail(nullptr, CMLBM_ERR_UNSUPPORTED, "the TMA-staged step does not cover slab handles");
    if (!(c.tau > 0.5) || !std::isfinite(c.tau)) return fail(nullptr, CMLBM_ERR_INVALID, "tau must be > 1/2");
    if (c.omega_bulk != 0.0 && !valid_omega(c.omega_bulk)) return fail(nullptr, CMLBM_ERR_INVALID, "omega_bulk must be 0 or in (0, 2)");
    if (!valid_omega(c.omega_3) || !valid_omega(c.omega_4)) return fail(nullptr, CMLBM_ERR_INVALID, "omega_3 and omega_4 must be in (0, 2)");
    if (!(c.smagorinsky_cs >= 0.0)) return fail(nullptr, CMLBM_ERR_INVALID, "smagorinsky_cs must be >= 0");
    if (c.van_driest_aplus != 0.0) {
        if (!(c.van_driest_aplus > 0.0) || !(c.van_driest_utau_over_nu > 0.0))
            return fail(nullptr, CMLBM_ERR_INVALID, "van Driest needs A+ > 0 and u_tau/nu > 0");
        if (c.bc[1] != CMLBM_BOUNCEBACK) return fail(nullptr, CMLBM_ERR_INVALID, "van Driest damping needs walls in y");
        if (c.smagorinsky_cs <= 0.0) return fail(nullptr, CMLBM_ERR_INVALID, "van Driest damping needs smagorinsky_cs > 0");
    }
    if (c.attractor != CMLBM_ATTRACTOR_MAXWELL && c.attractor != CMLBM_ATTRACTOR_FACTORIZED)
        return fail(nullptr, CMLBM_ERR_INVALID, "unknown attractor");
    if (c.reduced_compressibility && !(c.rho0 > 0.0)) return fail(nullptr, CMLBM_ERR_INVALID, "rho0 must be > 0");

    cmlbm* h = new (std::nothrow) cmlbm();
    if (!h) return fail(nullptr, CMLBM_ERR_NOMEM, "host allocation failed");
    h->cfg = c;
    h->D = (c.lattice == CMLBM_D3Q27) ? 3 : 2;
    h->Q = (h->D == 3) ? 27 : 9;
    h->esize = storage_size(c.storage);
    h->rsize = (c.storage == CMLBM_F64) ? 8 : 4;
    h->st = (cudaStream_t)c.stream;
    cm::Params& p = h->p;
    std::memset(&p, 0, sizeof(p));
    p.nx = c.nx;
    p.ny = c.ny;
    p.nz = c.nz;
    p.N = N;
    p.S = S;
    p.big = big ? 1 : 0;
    h->ghost = slab ? (size_t)c.nx * c.ny : 0;
    for (int a = 0; a < 3; ++a) p.bc[a] = c.bc[a];
    std::memcpy(p.uw, c.wall_velocity, sizeof(p.uw));
    p.tau0 = c.tau;
    p.omega_bulk = c.omega_bulk;
    p.omega3 = c.omega_3;
    p.omega4 = c.omega_4;
    p.cs = c.smagorinsky_cs;
    p.les = c.smagorinsky_cs > 0.0;
    p.vd = c.van_driest_aplus > 0.0;
    p.vd_aplus = c.van_driest_aplus;
    p.vd_utau_nu = c.van_driest_utau_over_nu;
    p.attractor = c.attractor;
    p.reduced = c.reduced_compressibility ? 1 : 0;
    p.rho0 = c.reduced_compressibility ? c.rho0 : 1.0;

    DeviceGuard g(c.device);
    if (!g.ok) {
        delete h;
        return fail(nullptr, CMLBM_ERR_CUDA, "cudaSetDevice failed");
    }
    const size_t bytes = (size_t)h->Q * (size_t)S * h->esize;
    for (int k = 0; k < 2; ++k) {
        if (grid_alloc(&h->buf[k], bytes) != cudaSuccess) {
            cudaGetLastError();
            cmlbm_destroy(h);
            return fail(nullptr, CMLBM_ERR_NOMEM, "cudaMalloc of the state buffers failed");
        }
    }
    if (cudaMalloc(&h->part, sizeof(double) * 5 * cm::kReduceMaxBlocks) != cudaSuccess ||
        cudaMalloc(&h->red, sizeof(double) * 5) != cudaSuccess || cudaMalloc(&h->flag, sizeof(int)) != cudaSuccess ||
        cudaMemset(h->flag, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cmlbm_destroy(h);
        return fail(nullptr, CMLBM_ERR_NOMEM, "cudaMalloc of the reduction buffers failed");
    }
    if (cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess) h->nsm = 1;
    if ((c.kernel == CMLBM_KERNEL_AUTO || big) && cm::pair_eligible(p, h->D, c.storage != CMLBM_F64)) p.pair = 1;
    const bool two_ok = cm::two_steps_eligible(p, h->D, c.storage == CMLBM_F32, slab);
    if (c.kernel == CMLBM_KERNEL_PAIR_TWO_STEPS && !two_ok) {
        cmlbm_destroy(h);
        return fail(nullptr, CMLBM_ERR_UNSUPPORTED,
                    "two steps per pass need D3Q27, FP32 storage, periodic x, nx a multiple of 64, nz >= 16, "
                    "no slab and the standard collision");
    }
    // opt-in only: measured slower than single steps of the pair kernel (see the header)
    if (c.kernel == CMLBM_KERNEL_PAIR_TWO_STEPS && two_ok) {
        p.pair = 1;
        h->two_steps = true;
    }
    if (c.kernel == CMLBM_KERNEL_PAIR) {
        if (!cm::pair_eligible(p, h->D, c.storage != CMLBM_F64)) {
            cmlbm_destroy(h);
            return fail(nullptr, CMLBM_ERR_UNSUPPORTED,
                        "the two-cells-per-thread step needs D3Q27, FP32/BF16/FP16 storage, periodic x and nx a "
                        "multiple of 64");
        }
        p.pair = 1;
    }
    if (c.kernel == CMLBM_KERNEL_TMA) {
        const bool eligible = h->D == 3 && c.storage != CMLBM_F64 && c.attractor == CMLBM_ATTRACTOR_MAXWELL &&
                              !c.reduced_compressibility;
        bool ok = eligible;
        for (int k = 0; k < 2 && ok; ++k) ok = cm::encode_tma_maps(h->buf[k], p, c.storage, h->maps[k][0], h->maps[k][1]);
        h->tma = ok;
        if (ok) {
            void* hf = nullptr;
            if (cudaHostAlloc(&hf, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                cmlbm_destroy(h);
                return fail(nullptr, CMLBM_ERR_NOMEM, "cudaHostAlloc of the pipeline flag mirror failed");
            }
            h->hflag = (volatile int*)hf;
            *h->hflag = 0;
        }
        if (!ok && c.kernel == CMLBM_KERNEL_TMA) {
            cmlbm_destroy(h);
            return fail(nullptr, CMLBM_ERR_UNSUPPORTED,
                        "the TMA-staged step needs D3Q27, FP32/BF16/FP16 storage, nx a multiple of 128 and the "
                        "standard collision");
        }
    }
    int rc = cmlbm_init(h, nullptr, nullptr, CMLBM_DEVICE);
    if (rc != CMLBM_OK) {
        std::string m = h->err;
        cmlbm_destroy(h);
        return fail(nullptr, rc, m);
    }
    cudaError_t e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) {
        cmlbm_destroy(h);
        return cuda_fail(nullptr, e, "initialisation");
    }
    *out = h;
    return CMLBM_OK;
}

void cmlbm_destroy(cmlbm_t* h) {
    if (!h) return;
    DeviceGuard g(h->cfg.device);
    cudaStreamSynchronize(h->st);
    if (h->inner) {
        cudaStreamSynchronize(h->inner);
        cudaStreamDestroy(h->inner);
    }
    if (h->ev_begin) cudaEventDestroy(h->ev_begin);
    if (h->ev_interior) cudaEventDestroy(h->ev_interior);
    drop_graphs(h);
    if (h->cap) cudaStreamDestroy(h->cap);
    cudaFree(h->buf[0]);
    cudaFree(h->buf[1]);
    cudaFree(h->force);
    cudaFree(h->part);
    cudaFree(h->red);
    cudaFree(h->stage);
    cudaFree(h->flag);
    cudaFree(h->turb);
    cudaFree(h->ring);
    if (h->hflag) cudaFreeHost((void*)h->hflag);
    delete h;
}

int cmlbm_set_stream(cmlbm_t* h, void* stream) {
    if (!h) return CMLBM_ERR_INVALID;
    h->st = (cudaStream_t)stream;
    return CMLBM_OK;
}

long long cmlbm_launch_count(const cmlbm_t* h) { return h ? h->launches : 0; }

int cmlbm_step_kernel(const cmlbm_t* h) {
    if (!h) return CMLBM_ERR_INVALID;
    if (h->tma) return CMLBM_KERNEL_TMA;
    if (h->two_steps) return CMLBM_KERNEL_PAIR_TWO_STEPS;
    return h->p.pair ? CMLBM_KERNEL_PAIR : CMLBM_KERNEL_DIRECT;
}

size_t cmlbm_state_bytes(const cmlbm_t* h) { return h ? (size_t)h->Q * (size_t)h->p.S * h->esize : 0; }

int cmlbm_set_force(cmlbm_t* h, const double uniform[3], const double* field, int where) {
    if (!h) return CMLBM_ERR_INVALID;
    DeviceGuard g(h->cfg.device);
    if (cudaError_t ej = join_interior(h); ej != cudaSuccess) return cuda_fail(h, ej, "interior join");
    drop_graphs(h);            // the captured steps carry the old force parameters
    for (int d = 0; d < 3; ++d) {
        const double v = uniform ? uniform[d] : 0.0;
        if (!std::isfinite(v)) return fail(h, CMLBM_ERR_INVALID, "uniform force must be finite");
        h->p.F[d] = v;
    }
    if (!field) {
        h->p.has_field = 0;
        return CMLBM_OK;
    }
    if (where != CMLBM_DEVICE && where != CMLBM_HOST) return fail(h, CMLBM_ERR_INVALID, "bad `where`");
    const long long n = 3 * h->p.N;
    if (!h->force) {
        if (grid_alloc(&h->force, h->rsize * (size_t)n) != cudaSuccess) {
            h->force = nullptr;
            cudaGetLastError();
            return fail(h, CMLBM_ERR_NOMEM, "cudaMalloc of the force field failed");
        }
    }
    const double* src = field;
    if (where == CMLBM_HOST) {
        int rc = ensure_stage(h);
        if (rc) return rc;
        cudaError_t e = cudaMemcpyAsync(h->stage, field, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, h->st);
        if (e != cudaSuccess) return cuda_fail(h, e, "force upload");
        src = h->stage;
    }
    ++h->launches;
    cudaError_t e = cm::launch_convert_force(src, h->force, n, h->cfg.storage == CMLBM_F64, h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "force conversion");
    if (where == CMLBM_HOST) {
        e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) return cuda_fail(h, e, "force upload");
    }
    h->p.has_field = 1;
    return CMLBM_OK;
}

// The device address of page-locked host memory that the CUDA runtime maps into the device's
// address space (cudaHostAlloc / cudaMallocHost, or cudaHostRegister with mapping): kernels read
// and write it directly over the host link, with no staging copy. nullptr for any other pointer
// (pageable memory goes through the device staging buffer and cudaMemcpyAsync).
static void* mapped_host(const void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

int cmlbm_init(cmlbm_t* h, const double* rho, const double* u, int where) {
    if (!h) return CMLBM_ERR_INVALID;
    if (where != CMLBM_DEVICE && where != CMLBM_HOST) return fail(h, CMLBM_ERR_INVALID, "bad `where`");
    DeviceGuard g(h->cfg.device);
    if (cudaError_t ej = join_interior(h); ej != cudaSuccess) return cuda_fail(h, ej, "interior join");
    const size_t N = (size_t)h->p.N;
    void* dst = own(h, h->buf[h->cur]);
    auto launch = [&](const double* r, const double* v, int z0, int nzc) {
        ++h->launches;
        return dispatch(h, [&](auto d, auto* s) {
            using S = std::remove_pointer_t<decltype(s)>;
            return cm::launch_init<decltype(d)::value, S>(dst, h->force, h->p, r, v, h->st, z0, nzc);
        });
    };
    const double* drho = rho;
    const double* du = u;
    const double* mrho = (const double*)mapped_host(rho);
    const double* mu = (const double*)mapped_host(u);
    if (where == CMLBM_HOST && (!rho || mrho) && (!u || mu)) {
        // page-locked fields: the init kernel reads them in place
        drho = mrho;
        du = mu;
    } else if (where == CMLBM_HOST && (rho || u)) {
        int rc = ensure_stage(h);
        if (rc) return rc;
        if (rho) {
            cudaError_t e = cudaMemcpyAsync(h->stage, rho, sizeof(double) * N, cudaMemcpyHostToDevice, h->st);
            if (e != cudaSuccess) return cuda_fail(h, e, "rho upload");
            drho = h->stage;
        }
        if (u) {
            cudaError_t e = cudaMemcpyAsync(h->stage + N, u, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, h->st);
            if (e != cudaSuccess) return cuda_fail(h, e, "u upload");
            du = h->stage + N;
        }
    }
    cudaError_t e = launch(drho, du, 0, h->p.nz);
    if (e != cudaSuccess) return cuda_fail(h, e, "init kernels");
    if (where == CMLBM_HOST) {
        e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) return cuda_fail(h, e, "init");
    }
    return CMLBM_OK;
}

int cmlbm_step(cmlbm_t* h, int nsteps) {
    if (!h) return CMLBM_ERR_INVALID;
    if (nsteps < 0) return fail(h, CMLBM_ERR_INVALID, "nsteps must be >= 0");
    DeviceGuard g(h->cfg.device);
    if (int rc = check_flag(h)) return rc;
    if (h->boundary_done) return fail(h, CMLBM_ERR_INVALID, "a split step waits for its interior part");
    if (cudaError_t ej = join_interior(h); ej != cudaSuccess) return cuda_fail(h, ej, "interior join");
    const bool stepped = nsteps > 0;
    if (nsteps >= 2 && h->two_steps && !h->ring) {
        const size_t bytes = (size_t)(cm::kTwoStepRing + 2) * h->p.nx * h->p.ny * h->Q * h->esize;
        if (grid_alloc(&h->ring, bytes) != cudaSuccess) {
            cudaGetLastError();
            h->ring = nullptr;
            h->two_steps = false;      // no room for the ring: single steps
            drop_graphs(h);
        }
    }
    // pairs of steps as graph replays (one graph launch instead of two or more kernel launches)
    if (nsteps >= 2 && h->graphs && !h->tma) {
        if (!h->gexec[h->cur] && capture_two_steps(h, h->cur, &h->gexec[h->cur]) != cudaSuccess) {
            cudaGetLastError();
            h->gexec[h->cur] = nullptr;
            h->graphs = false;
        }
        for (; nsteps >= 2 && h->gexec[h->cur]; nsteps -= 2) {
            cudaError_t e = cudaGraphLaunch(h->gexec[h->cur], h->st);
            if (e != cudaSuccess) return cuda_fail(h, e, "step graph launch");
            if (h->two_steps) {
                h->launches += h->pass_launches;
                h->cur ^= 1;
                if (nsteps >= 4 && !h->gexec[h->cur] && capture_two_steps(h, h->cur, &h->gexec[h->cur]) != cudaSuccess) {
                    cudaGetLastError();
                    h->gexec[h->cur] = nullptr;
                }
            } else {
                h->launches += 2;
            }
        }
    }
    // without graphs: two-step passes launched directly
    for (; nsteps >= 2 && h->two_steps; nsteps -= 2) {
        cudaError_t e = enqueue_two_steps(h, h->cur);
        if (e != cudaSuccess) return cuda_fail(h, e, "two-step pass");
        h->cur ^= 1;
    }
    for (int k = 0; k < nsteps; ++k) {
        cudaError_t e = do_step(h, h->buf[h->cur], h->buf[1 - h->cur]);
        if (e != cudaSuccess) return cuda_fail(h, e, "step kernel");
        h->cur ^= 1;
    }
    if (stepped) {
        cudaError_t e = mirror_flag(h);
        if (e != cudaSuccess) return cuda_fail(h, e, "pipeline flag copy");
    }
    return CMLBM_OK;
}

int cmlbm_step_buffers(cmlbm_t* h, const void* src, void* dst) {
    if (!h) return CMLBM_ERR_INVALID;
    if (!src || !dst || src == dst) return fail(h, CMLBM_ERR_INVALID, "src and dst must be distinct device buffers");
    DeviceGuard g(h->cfg.device);
    if (int rc = check_flag(h)) return rc;
    if (cudaError_t ej = join_interior(h); ej != cudaSuccess) return cuda_fail(h, ej, "interior join");
    cudaError_t e = do_step(h, src, dst);
    if (e != cudaSuccess) return cuda_fail(h, e, "step kernel");
    e = mirror_flag(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "pipeline flag copy");
    return CMLBM_OK;
}

int cmlbm_step_split(cmlbm_t* h, int parts) {
    if (!h) return CMLBM_ERR_INVALID;
    if (parts < CMLBM_SPLIT_BOUNDARY || parts > CMLBM_SPLIT_BOTH) return fail(h, CMLBM_ERR_INVALID, "bad parts");
    if (h->tma || h->two_steps)
        return fail(h, CMLBM_ERR_UNSUPPORTED, "split steps use the direct or two-cells-per-thread kernel");
    if (parts == CMLBM_SPLIT_INTERIOR && !h->boundary_done)
        return fail(h, CMLBM_ERR_INVALID, "the interior part of a split step needs its boundary part first");
    if (parts != CMLBM_SPLIT_INTERIOR && h->boundary_done)
        return fail(h, CMLBM_ERR_INVALID, "the interior part of the previous split step is still to come");
    DeviceGuard g(h->cfg.device);
    if (!h->inner) {
        // the interior runs at the lowest stream priority, so that the boundary planes and the
        // face exchange, issued on a stream of higher priority, are dispatched ahead of its blocks
        int lowest = 0, highest = 0;
        cudaError_t e = cudaDeviceGetStreamPriorityRange(&lowest, &highest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->inner, cudaStreamNonBlocking, lowest);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_begin, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_interior, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(h, e, "split-step stream");
    }
    const int nz = h->p.nz;
    const void* src = h->buf[h->cur];
    void* dst = h->buf[1 - h->cur];
    cudaError_t e = cudaSuccess;
    if (parts & CMLBM_SPLIT_BOUNDARY) {
        // the interior starts after everything issued so far on the handle's stream (the
        // previous step's boundary planes and the face exchange that followed it)
        e = cudaEventRecord(h->ev_begin, h->st);
        // the boundary planes pull from the planes next to them, written by the previous interior
        if (e == cudaSuccess) e = join_interior(h);
        if (e == cudaSuccess) e = do_step_planes(h, src, dst, 0, 1, h->st);
        if (e == cudaSuccess && nz > 1) e = do_step_planes(h, src, dst, nz - 1, 1, h->st);
        h->boundary_done = e == cudaSuccess;
    }
    if (e == cudaSuccess && (parts & CMLBM_SPLIT_INTERIOR)) {
        e = cudaStreamWaitEvent(h->inner, h->ev_begin, 0);
        if (e == cudaSuccess && nz > 2) {
            e = do_step_planes(h, src, dst, 1, nz - 2, h->inner);
            if (e == cudaSuccess) e = cudaEventRecord(h->ev_interior, h->inner);
            if (e == cudaSuccess) h->interior_pending = true;
        }
        h->boundary_done = false;
        if (e == cudaSuccess) h->cur ^= 1;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "split step");
    return CMLBM_OK;
}

int cmlbm_moments_of(cmlbm_t* h, const void* state, double* rho, double* u) {
    if (!h) return CMLBM_ERR_INVALID;
    if (!state) return fail(h, CMLBM_ERR_INVALID, "state is NULL");
    if (!rho && !u) return CMLBM_OK;
    DeviceGuard g(h->cfg.device);
    if (int rc = check_flag(h)) return rc;
    if (cudaError_t ej = join_interior(h); ej != cudaSuccess) return cuda_fail(h, ej, "interior join");
    cudaError_t e = do_moments(h, state, rho, u);
    if (e != cudaSuccess) return cuda_fail(h, e, "moments kernel");
    return CMLBM_OK;
}

int cmlbm_moments(cmlbm_t* h, double* rho, double* u, int where) {
    if (!h) return CMLBM_ERR_INVALID;
    if (where != CMLBM_DEVICE && where != CMLBM_HOST) return fail(h, CMLBM_ERR_INVALID, "bad `where`");
    if (!rho && !u) return CMLBM_OK;
    DeviceGuard g(h->cfg.device);
    if (where == CMLBM_DEVICE) return cmlbm_moments_of(h, h->buf[h->cur], rho, u);
    if (int rc = check_flag(h)) return rc;
    if (cudaError_t ej = join_interior(h); ej != cudaSuccess) return cuda_fail(h, ej, "interior join");

    double* mrho = (double*)mapped_host(rho);
    double* mu = (double*)mapped_host(u);
    if ((!rho || mrho) && (!u || mu)) {
        // page-locked outputs: the moments kernel writes them in place
        cudaError_t e = do_moments(h, h->buf[h->cur], mrho, mu);
        if (e != cudaSuccess) return cuda_fail(h, e, "moments kernel");
        e = cudaStreamSynchronize(h->st);
        if (e != cudaSuccess) return cuda_fail(h, e, "moments");
        return check_flag(h);
    }
    int rc = ensure_stage(h);
    if (rc) return rc;
    const size_t N = (size_t)h->p.N;
    cudaError_t e = do_moments(h, h->buf[h->cur], h->stage, h->stage + N);
    if (e != cudaSuccess) return cuda_fail(h, e, "moments kernel");
    if (rho && (e = cudaMemcpyAsync(rho, h->stage, sizeof(double) * N, cudaMemcpyDeviceToHost, h->st)) != cudaSuccess)
        return cuda_fail(h, e, "rho download");
    if (u && (e = cudaMemcpyAsync(u, h->stage + N, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, h->st)) != cudaSuccess)
        return cuda_fail(h, e, "u download");
    e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "moments");
    return check_flag(h);
}

int cmlbm_reduce(cmlbm_t* h, double out[5]) {
    if (!h || !out) return CMLBM_ERR_INVALID;
    DeviceGuard g(h->cfg.device);
    if (cudaError_t ej = join_interior(h); ej != cudaSuccess) return cuda_fail(h, ej, "interior join");
    h->launches += 2;
    cudaError_t e = dispatch(h, [&](auto d, auto* s) {
        using S = std::remove_pointer_t<decltype(s)>;
        return cm::launch_reduce<decltype(d)::value, S>(own(h, h->buf[h->cur]), h->force, h->p, h->part, h->red, h->st);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "reduction kernels");
    e = cudaMemcpyAsync(out, h->red, sizeof(double) * 5, cudaMemcpyDeviceToHost, h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "reduction download");
    e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "reduction");
    if (int rc = check_flag(h)) return rc;
    for (int k = 0; k < 5; ++k)
        if (!std::isfinite(out[k])) return fail(h, CMLBM_ERR_DIVERGED, "non-finite value in the reductions");
    return CMLBM_OK;
}

int cmlbm_get_state(cmlbm_t* h, void* dst, size_t bytes, int where) {
    if (!h || !dst) return CMLBM_ERR_INVALID;
    if (bytes != cmlbm_state_bytes(h)) return fail(h, CMLBM_ERR_INVALID, "bytes must equal cmlbm_state_bytes");
    if (where != CMLBM_DEVICE && where != CMLBM_HOST) return fail(h, CMLBM_ERR_INVALID, "bad `where`");
    DeviceGuard g(h->cfg.device);
    if (int rc = check_flag(h)) return rc;
    if (cudaError_t ej = join_interior(h); ej != cudaSuccess) return cuda_fail(h, ej, "interior join");
    cudaError_t e = cudaMemcpyAsync(dst, h->buf[h->cur], bytes, where == CMLBM_HOST ? cudaMemcpyDeviceToHost
                                                                                   : cudaMemcpyDeviceToDevice, h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "state copy");
    if (where == CMLBM_HOST && (e = cudaStreamSynchronize(h->st)) != cudaSuccess) return cuda_fail(h, e, "state copy");
    return where == CMLBM_HOST ? check_flag(h) : CMLBM_OK;
}

int cmlbm_set_state(cmlbm_t* h, const void* src, size_t bytes, int where) {
    if (!h || !src) return CMLBM_ERR_INVALID;
    if (bytes != cmlbm_state_bytes(h)) return fail(h, CMLBM_ERR_INVALID, "bytes must equal cmlbm_state_bytes");
    if (where != CMLBM_DEVICE && where != CMLBM_HOST) return fail(h, CMLBM_ERR_INVALID, "bad `where`");
    if (h->boundary_done) return fail(h, CMLBM_ERR_INVALID, "a split step waits for its interior part");
    DeviceGuard g(h->cfg.device);
    if (cudaError_t ej = join_interior(h); ej != cudaSuccess) return cuda_fail(h, ej, "interior join");
    cudaError_t e = cudaMemcpyAsync(h->buf[h->cur], src, bytes, where == CMLBM_HOST ? cudaMemcpyHostToDevice
                                                                                   : cudaMemcpyDeviceToDevice, h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "state copy");
    if (where == CMLBM_HOST && (e = cudaStreamSynchronize(h->st)) != cudaSuccess) return cuda_fail(h, e, "state copy");
    return CMLBM_OK;
}

int cmlbm_turbulence_force(cmlbm_t* h, double cs) {
    if (!h) return CMLBM_ERR_INVALID;
    if (!(cs >= 0.0) || !std::isfinite(cs)) return fail(h, CMLBM_ERR_INVALID, "cs must be finite and >= 0");
    if (h->p.bc[0] || h->p.bc[1] || h->p.bc[2])
        return fail(h, CMLBM_ERR_UNSUPPORTED, "turbulence forcing needs periodic boundaries");
    if (h->p.big) return fail(h, CMLBM_ERR_UNSUPPORTED, "turbulence forcing needs 27*N < 2^32 (32-bit element offsets)");
    DeviceGuard g(h->cfg.device);
    if (cudaError_t ej = join_interior(h); ej != cudaSuccess) return cuda_fail(h, ej, "interior join");
    const size_t N = (size_t)h->p.N;
    if (!h->force || !h->p.has_field) drop_graphs(h);   // the steps will read a (new) force field
    if (!h->force && grid_alloc(&h->force, h->rsize * 3 * N) != cudaSuccess) {
        h->force = nullptr;
        cudaGetLastError();
        return fail(h, CMLBM_ERR_NOMEM, "cudaMalloc of the force field failed");
    }
    if (!h->turb && grid_alloc(&h->turb, h->rsize * 10 * N) != cudaSuccess) {
        h->turb = nullptr;
        cudaGetLastError();
        return fail(h, CMLBM_ERR_NOMEM, "cudaMalloc of the turbulence scratch failed");
    }
    h->launches += 3;
    cudaError_t e = dispatch(h, [&](auto d, auto* s) {
        using S = std::remove_pointer_t<decltype(s)>;
        return cm::launch_turbulence_force<decltype(d)::value, S>(h->buf[h->cur], h->force, h->p, cs, h->turb, h->st);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "turbulence forcing kernels");
    h->p.has_field = 1;
    return CMLBM_OK;
}

int cmlbm_step_filtered(cmlbm_t* h, int nsteps, double cs) {
    if (!h) return CMLBM_ERR_INVALID;
    if (nsteps < 0) return fail(h, CMLBM_ERR_INVALID, "nsteps must be >= 0");
    for (int k = 0; k < nsteps; ++k) {
        int rc = cmlbm_turbulence_force(h, cs);
        if (rc) return rc;
        rc = cmlbm_step(h, 1);
        if (rc) return rc;
    }
    return CMLBM_OK;
}

static int adjoint_supported(cmlbm* h) {
    if (h->ghost) return fail(h, CMLBM_ERR_UNSUPPORTED, "the adjoint does not cover slab handles");
    if (h->p.big) return fail(h, CMLBM_ERR_UNSUPPORTED, "the adjoint needs 27*N < 2^32 (32-bit element offsets)");
    if (h->cfg.storage != CMLBM_F64 && h->cfg.storage != CMLBM_F32)
        return fail(h, CMLBM_ERR_UNSUPPORTED, "the adjoint needs F64 or F32 storage");
    if (h->p.les || h->p.attractor != 0 || h->p.reduced)
        return fail(h, CMLBM_ERR_UNSUPPORTED, "the adjoint supports the Maxwellian attractor without eddy viscosity");
    return CMLBM_OK;
}

int cmlbm_adjoint_terminal(cmlbm_t* h, const void* state, const double* dLdu, const double* dLdrho, void* lambda,
                           double* dLdF) {
    if (!h) return CMLBM_ERR_INVALID;
    if (!state || !dLdu || !lambda || !dLdF) return fail(h, CMLBM_ERR_INVALID, "NULL argument");
    int rc = adjoint_supported(h);
    if (rc) return rc;
    DeviceGuard g(h->cfg.device);
    if (cudaError_t ej = join_interior(h); ej != cudaSuccess) return cuda_fail(h, ej, "interior join");
    ++h->launches;
    cudaError_t e;
    if (h->D == 3)
        e = (h->cfg.storage == CMLBM_F64)
                ? cm::launch_adjoint_terminal<3, double>(state, h->force, h->p, dLdu, dLdrho, lambda, dLdF, h->st)
                : cm::launch_adjoint_terminal<3, float>(state, h->force, h->p, dLdu, dLdrho, lambda, dLdF, h->st);
    else
        e = (h->cfg.storage == CMLBM_F64)
                ? cm::launch_adjoint_terminal<2, double>(state, h->force, h->p, dLdu, dLdrho, lambda, dLdF, h->st)
                : cm::launch_adjoint_terminal<2, float>(state, h->force, h->p, dLdu, dLdrho, lambda, dLdF, h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint terminal kernel");
    return CMLBM_OK;
}

static int step_adjoint(cmlbm* h, const void* state, const void* lambda_in, void* lambda_out, double* dLdF,
                        void* seg, int acc) {
    if (!h) return CMLBM_ERR_INVALID;
    if (!state || !lambda_in || !lambda_out || !dLdF) return fail(h, CMLBM_ERR_INVALID, "NULL argument");
    if (acc != 0 && !seg) return fail(h, CMLBM_ERR_INVALID, "seg is NULL");
    if (lambda_in == lambda_out) return fail(h, CMLBM_ERR_INVALID, "lambda_in and lambda_out must not alias");
    int rc = adjoint_supported(h);
    if (rc) return rc;
    DeviceGuard g(h->cfg.device);
    if (cudaError_t ej = join_interior(h); ej != cudaSuccess) return cuda_fail(h, ej, "interior join");
    ++h->launches;
    cudaError_t e;
    if (h->D == 3)
        e = (h->cfg.storage == CMLBM_F64)
                ? cm::launch_adjoint_step<3, double>(state, h->force, h->p, lambda_in, lambda_out, dLdF, seg, acc, h->st)
                : cm::launch_adjoint_step<3, float>(state, h->force, h->p, lambda_in, lambda_out, dLdF, seg, acc, h->st);
    else
        e = (h->cfg.storage == CMLBM_F64)
                ? cm::launch_adjoint_step<2, double>(state, h->force, h->p, lambda_in, lambda_out, dLdF, seg, acc, h->st)
                : cm::launch_adjoint_step<2, float>(state, h->force, h->p, lambda_in, lambda_out, dLdF, seg, acc, h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint step kernel");
    return CMLBM_OK;
}

int cmlbm_step_adjoint(cmlbm_t* h, const void* state, const void* lambda_in, void* lambda_out, double* dLdF) {
    return step_adjoint(h, state, lambda_in, lambda_out, dLdF, nullptr, 0);
}

int cmlbm_step_adjoint_segment(cmlbm_t* h, const void* state, const void* lambda_in, void* lambda_out, void* seg,
                               double* dLdF, int fold) {
    return step_adjoint(h, state, lambda_in, lambda_out, dLdF, seg, fold ? 2 : 1);
}

// ---- slab decomposition: face messages ----------------------------------------------------
// A face message is 9 direction planes of one z-plane: directions 9 (e_z + 1) + 0..8, i.e.
// 0..8 (e_z = -1) or 18..26 (e_z = +1), each nx*ny contiguous values. One strided 2D copy
// moves the 9 planes (source pitch = the buffer's direction stride).
size_t cmlbm_halo_bytes(const cmlbm_t* h) { return h && h->ghost ? (size_t)9 * h->ghost * h->esize : 0; }

static int halo_copy(cmlbm* h, int face, void* msg, const void* cmsg, int where, bool pack) {
    if (!h) return CMLBM_ERR_INVALID;
    if (!h->ghost) return fail(h, CMLBM_ERR_INVALID, "the handle is not a slab (bc[2] != CMLBM_HALO)");
    if (face != CMLBM_FACE_BOTTOM && face != CMLBM_FACE_TOP) return fail(h, CMLBM_ERR_INVALID, "bad face");
    if (where != CMLBM_DEVICE && where != CMLBM_HOST) return fail(h, CMLBM_ERR_INVALID, "bad `where`");
    if (pack ? !msg : !cmsg) return fail(h, CMLBM_ERR_INVALID, "message buffer is NULL");
    DeviceGuard g(h->cfg.device);
    const size_t plane = h->ghost;                 // nx * ny
    const size_t pitch = (size_t)h->p.S * h->esize;
    const size_t width = plane * h->esize;
    // buffer plane index (0 = ghost below, 1 .. nz own planes, nz + 1 = ghost above)
    int dir0, zplane;
    if (pack) {
        dir0 = (face == CMLBM_FACE_TOP) ? 18 : 0;            // populations leaving through the face
        zplane = (face == CMLBM_FACE_TOP) ? h->p.nz : 1;
    } else {
        dir0 = (face == CMLBM_FACE_BOTTOM) ? 18 : 0;         // populations entering through the face
        zplane = (face == CMLBM_FACE_BOTTOM) ? 0 : h->p.nz + 1;
    }
    char* state = (char*)h->buf[h->cur] + ((size_t)dir0 * h->p.S + (size_t)zplane * plane) * h->esize;
    cudaError_t e;
    if (pack)
        e = cudaMemcpy2DAsync(msg, width, state, pitch, width, 9,
                              where == CMLBM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->st);
    else
        e = cudaMemcpy2DAsync(state, pitch, cmsg, width, width, 9,
                              where == CMLBM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, pack ? "face pack" : "face unpack");
    if (where == CMLBM_HOST && (e = cudaStreamSynchronize(h->st)) != cudaSuccess)
        return cuda_fail(h, e, pack ? "face pack" : "face unpack");
    return CMLBM_OK;
}

int cmlbm_halo_pack(cmlbm_t* h, int face, void* out, int where) { return halo_copy(h, face, out, nullptr, where, true); }

int cmlbm_halo_unpack(cmlbm_t* h, int face, const void* in, int where) {
    return halo_copy(h, face, nullptr, in, where, false);
}

}  // extern "C"
