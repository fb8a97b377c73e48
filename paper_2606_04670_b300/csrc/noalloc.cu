// lip_estimate_M_noalloc: the Lipschitz-constant estimate without any allocation.
//
// The ordinary entry points keep their working memory in the handle and grow it with
// cudaMalloc.  Some callers cannot do that: a plugin running inside a host application
// whose own allocator has already reserved the GPU's memory (a cudaMalloc from us would
// fail or fragment that pool), or a latency-bound loop that cannot absorb the device-wide
// synchronisation that cudaFree implies.  This entry point takes the data straight from
// the caller's device buffers, writes its result into a caller buffer, and keeps its
// working memory in the fixed array below, which every GPU that loads the library holds
// until the process exits.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "launch.h"

namespace lip {
lip_status set_error(lip_status s, const char* msg);
}

using namespace lip;

namespace {

constexpr int64_t NA_TILE = 512;   // the estimate kernel's tile (checked against the kernel at run time)
constexpr int64_t NA_POINTS = ((int64_t)LIP_NOALLOC_N_MAX + NA_TILE - 1) / NA_TILE * NA_TILE;
constexpr int64_t NA_LAYOUT_BYTES = (NA_POINTS * (D_MAX + 1) * 4 + 255) / 256 * 256;
constexpr int64_t NA_TILES = NA_POINTS / NA_TILE;
constexpr int64_t NA_CAND_BYTES = (NA_TILES * NA_TILES * 16 + 255) / 256 * 256;
constexpr int64_t NA_STATE_BYTES = 256;
constexpr int64_t NA_LIST_BYTES = (NA_TILES * NA_TILES * 4 + 255) / 256 * 256;
constexpr int64_t NA_BYTES = NA_LAYOUT_BYTES + NA_CAND_BYTES + NA_STATE_BYTES + NA_LIST_BYTES;   // about 4.4 MB (d up to 32)

// Working memory of every lip_estimate_M_noalloc call on this device: the FP32 point
// layout, one candidate record per tile pair, and the exact selection's device words and
// list of tile pairs.  Host code must not pass this
// name to a kernel (on the host it only stands for the symbol); it uses the address
// obtained from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_addr[MAX_DEVICES] = {};
unsigned long long g_ctx_id[MAX_DEVICES] = {};    // context the address belongs to (0: none yet)

// The driver's context queries, reached through the runtime so that the library does not
// link the driver library itself (it must load on machines without a GPU driver).
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
bool g_ctx_fns_looked_up = false;

// Identifier of the context current on this thread, or 0 when none is current (or the
// driver cannot say).
unsigned long long current_context_id() {
    if (!g_ctx_fns_looked_up) {
        g_ctx_fns_looked_up = true;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        void* f1 = nullptr;
        void* f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
        }
        cudaGetLastError();
    }
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != 0 || !ctx) return 0;
    if (g_ctx_get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of g_noalloc_scratch on the current device.  It is looked up once per
// device and context: cudaDeviceReset destroys the device's primary context, the module
// is loaded again in the next one and the array may move, so a new context id triggers a
// new lookup.  (Without the driver's context id the address is looked up on every call.)
lip_status scratch_address(int dev, void** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (dev < 0 || dev >= MAX_DEVICES) return set_error(LIP_ERR_UNSUPPORTED, "device ordinal beyond 63");
    const unsigned long long ctx = current_context_id();
    if (!g_addr[dev] || ctx == 0 || ctx != g_ctx_id[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char buf[256];
            snprintf(buf, sizeof buf, "cudaGetSymbolAddress(g_noalloc_scratch): %s", cudaGetErrorString(e));
            g_addr[dev] = nullptr;
            return set_error(LIP_ERR_CUDA, buf);
        }
        g_addr[dev] = p;
        // the lookup made the device's context current if none was
        g_ctx_id[dev] = ctx != 0 ? ctx : current_context_id();
    }
    *out = g_addr[dev];
    return LIP_OK;
}

lip_status launch_fail(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return set_error(e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver ? LIP_ERR_NO_DEVICE : LIP_ERR_CUDA,
                     buf);
}

}  // namespace

extern "C" lip_status lip_estimate_M_noalloc(const float* X, const float* y, int64_t N, int32_t d, int32_t norm,
                                             const double* w, double* out, void* stream) {
    if (!X || !y || !out) return set_error(LIP_ERR_ARG, "X, y or out is NULL");
    if (N < 1 || N > LIP_NOALLOC_N_MAX) {
        char buf[128];
        snprintf(buf, sizeof buf, "N = %lld is outside [1, %d], the fixed capacity of lip_estimate_M_noalloc",
                 (long long)N, LIP_NOALLOC_N_MAX);
        return set_error(LIP_ERR_ARG, buf);
    }
    if (d < 1 || d > D_MAX) return set_error(LIP_ERR_ARG, "d is outside [1, LIP_D_MAX]");
    if (norm < LIP_L1 || norm > LIP_LINF) return set_error(LIP_ERR_ARG, "norm is not L1/L2/Linf");
    if (w)
        for (int i = 0; i < d; ++i)
            if (!(w[i] > 0.0) || !std::isfinite(w[i])) return set_error(LIP_ERR_ARG, "w entries must be finite and > 0");
    if (estimate_tile_points() != NA_TILE) return set_error(LIP_ERR_UNSUPPORTED, "estimate tile size changed");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return launch_fail(e, "cudaGetDevice");
    void* base = nullptr;
    lip_status s = scratch_address(dev, &base);
    if (s != LIP_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    const int64_t nb = (N + NA_TILE - 1) / NA_TILE;
    const int64_t pts = nb * NA_TILE;
    const int nch = d + 1;
    char* lay = static_cast<char*>(base);
    float4* cand = reinterpret_cast<float4*>(static_cast<char*>(base) + NA_LAYOUT_BYTES);
    EstExactState* state = reinterpret_cast<EstExactState*>(static_cast<char*>(base) + NA_LAYOUT_BYTES + NA_CAND_BYTES);

    // Every byte read below is written first by this call: the layout covers [0, pts)
    // (data, then padding) and the candidate pass writes every tile pair it later reads.
    HotParams Hp{};
    Hp.X0 = X;
    Hp.y0 = y;
    Hp.k0 = 0;
    Hp.k1 = N;
    Hp.d = d;
    Hp.C = 0;
    Hp.dl = d;
    Hp.nch = nch;
    Hp.aux = 0;
    double wd[D_MAX];
    for (int j = 0; j < D_MAX; ++j) wd[j] = (w && j < d) ? w[j] : 1.0;
    const bool weighted = est_weighted(wd, d);
    for (int j = 0; j < D_MAX; ++j) {
        Hp.perm[j] = j;
        Hp.scale[j] = est_layout_scale(wd, j, weighted);
    }
    Hp.hot = lay;
    Hp.err = nullptr;
    EstFinalParams F{};
    F.cand = cand;
    F.nb = N < 2 ? 0 : (int)nb;
    F.X0 = X;
    F.y0 = y;
    F.d = d;
    F.norm = norm;
    F.elem_bytes = 4;
    for (int j = 0; j < D_MAX; ++j) F.w[j] = (w && j < d) ? w[j] : 1.0;
    F.out = out;
    F.lay = reinterpret_cast<const float4*>(lay);
    F.N = N;
    F.weighted = weighted;
    F.state = state;
    F.list = reinterpret_cast<unsigned*>(static_cast<char*>(base) + NA_LAYOUT_BYTES + NA_CAND_BYTES + NA_STATE_BYTES);
    if (N >= 2) {
        if ((e = launch_estimate_layout(4, Hp, st)) != cudaSuccess) return launch_fail(e, "estimate layout");
        if ((e = launch_pad_hot(4, lay, N, pts, nch, d, st)) != cudaSuccess) return launch_fail(e, "estimate padding");
        EstParams P{};
        P.lay = reinterpret_cast<const float4*>(lay);
        P.N = N;
        P.nb = (int)nb;
        P.cand = cand;
        P.weighted = weighted;
        for (int j = 0; j < d; ++j) P.w[j] = (float)wd[j];
        if ((e = launch_estimate(norm, d, P, st)) != cudaSuccess) return launch_fail(e, "estimate kernel");
    }
    if ((e = launch_estimate_final(F, st)) != cudaSuccess) return launch_fail(e, "estimate final");
    return LIP_OK;
}
