// he_noalloc.cu -- he_conv_layer_noalloc: the Conv layer call with no device
// allocation on its path.
//
// he_conv_layer transforms coefficient-domain inputs into the params'
// workspace, which the library cudaMallocs at model load and which caps the
// batch of a call.  Some callers cannot have the library allocate device
// memory for them at all: a serving loop that has split its whole HBM budget
// between requests up front, or a process whose device memory is owned by an
// outside allocator, must not see cudaMalloc (which can fail under memory
// pressure, and can synchronize the device) when a larger batch comes in.
// This entry point keeps that transform's scratch in a fixed array compiled
// into the library instead.
#include <cstdio>
#include <mutex>

#include "he_internal.h"

namespace {

// The scratch: forward-NTT images of a call's inputs, B*G*2*L*N words at most.
constexpr size_t kScratchWords = (size_t)2 * 1024 * 1024;  // 8 MiB
static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

// Device address of g_noalloc_scratch per device (the host-side symbol is
// only a stand-in), looked up once per device.
std::mutex g_mu;
uint32_t *g_addr[64] = {};

struct Guard {
    int prev = -1;
    bool ok = false;
    explicit Guard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~Guard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" he_status he_conv_layer_noalloc(he_params_t p, he_filters_t f, const uint32_t *d_in, int in_domain,
                                           uint32_t *d_out, int out_mode, uint32_t B, void *stream) {
    if (!p || !f || !d_in || !d_out) return he_fail(HE_ERR_ARG, "NULL argument");
    if (p->device == HE_DEVICE_NONE) return he_fail(HE_ERR_ARG, "params were created without a device");
    if (p->device < 0 || p->device >= 64) return he_fail(HE_ERR_ARG, "device ordinal out of range");
    if (f->kind != HE_KIND_CONV || f->p != p) return he_fail(HE_ERR_ARG, "filters are not a Conv bank of these params");
    if (f->masked) return he_fail(HE_ERR_ARG, "a masked bank is evaluated by he_conv_layer_masked");
    if (in_domain != HE_COEFF && in_domain != HE_NTT) return he_fail(HE_ERR_ARG, "bad in_domain");
    if (out_mode != HE_OUT_EXTRACTED && out_mode != HE_OUT_PER_CHANNEL && out_mode != HE_OUT_EXTRACTED_UNFOLDED)
        return he_fail(HE_ERR_ARG, "bad out_mode");
    if (B == 0) return he_fail(HE_ERR_ARG, "B must be >= 1");
    if (((uintptr_t)d_in & 15u) || ((uintptr_t)d_out & 15u)) return he_fail(HE_ERR_ARG, "buffers must be 16-byte aligned");
    const he_conv_layout &lay = f->lay;
    const size_t nin = (size_t)B * lay.G * 2u * p->L * p->N;
    const size_t nout = (size_t)B * (out_mode == HE_OUT_PER_CHANNEL ? f->desc.co : lay.H) * 2u * p->L * p->N;
    if (d_in < d_out + nout && d_out < d_in + nin) return he_fail(HE_ERR_ARG, "d_in and d_out overlap");
    if (in_domain == HE_COEFF && nin > kScratchWords) {
        char msg[160];
        snprintf(msg, sizeof(msg), "inputs need %zu scratch words, above the fixed %zu (8 MiB); use he_conv_layer", nin,
                 kScratchWords);
        return he_fail(HE_ERR_ARG, msg);
    }
    Guard g(p->device);
    if (!g.ok) return he_fail(HE_ERR_CUDA, "cannot select the params' device");
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t *x = d_in;
    if (in_domain == HE_COEFF) {
        uint32_t *scratch = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_mu);
            if (!g_addr[p->device]) {
                void *a = nullptr;
                const cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
                if (e != cudaSuccess) return he_fail(HE_ERR_CUDA, cudaGetErrorString(e));
                g_addr[p->device] = static_cast<uint32_t *>(a);
            }
            scratch = g_addr[p->device];
        }
        // the transform overwrites every scratch word it later reads: nothing
        // needs clearing between calls
        cudaError_t e = he_launch_ntt(p->ring, d_in, scratch, (uint32_t)(nin / p->N), false, st);
        if (e != cudaSuccess) return he_fail(HE_ERR_CUDA, cudaGetErrorString(e));
        x = scratch;
    }
    cudaError_t e = f->bank_s ? he_launch_conv(p->ring, f->desc, lay, f->logTS, f->lcs, 0u, f->bank_s, x, d_out, out_mode, B, st)
                              : he_launch_conv(p->ring, f->desc, lay, f->logTS, f->lcs, f->tc, f->bank, x, d_out, out_mode, B, st);
    if (e != cudaSuccess) return he_fail(HE_ERR_CUDA, cudaGetErrorString(e));
    return HE_OK;
}
