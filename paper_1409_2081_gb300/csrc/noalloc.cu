// Edge extraction for callers that cannot allocate device memory.  The
// paper has no counterpart.
//
// Same computation as hfcr_build_edges (sorted unique undirected edges of a
// triangle list), but every scratch buffer lives in one file-scope device
// array instead of a context's cudaMalloc'ed memory.  The array is sized for
// NOALLOC_MAX_TRIS triangles and, like any __device__ variable, occupies
// that much memory on every GPU that loads the library, until the process
// exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace hfcr {
void set_noctx_error(const std::string &msg);
}

namespace {

// HFCR_ERR_CUDA with the failing call's message for hfcr_last_error(NULL)
hfcr_status cuda_fail(const char *what, cudaError_t e) {
    hfcr::set_noctx_error(std::string("hfcr_build_edges_noalloc: ") + what + " failed: " +
                          cudaGetErrorString(e));
    return HFCR_ERR_CUDA;
}

constexpr int NOALLOC_MAX_TRIS = 1 << 16;
constexpr int NOALLOC_KEYS = 3 * NOALLOC_MAX_TRIS;              // one key per half-edge
constexpr int NOALLOC_HIST_BLOCKS = (NOALLOC_KEYS + 2047) / 2048 + 2;
constexpr size_t OFF_KEYS = 0;
constexpr size_t OFF_KEYS_ALT = OFF_KEYS + 8ull * NOALLOC_KEYS;
constexpr size_t OFF_FLAGS = OFF_KEYS_ALT + 8ull * NOALLOC_KEYS;
constexpr size_t OFF_HIST = OFF_FLAGS + 4ull * NOALLOC_KEYS;
constexpr size_t OFF_WORDS = OFF_HIST + 4ull * 256 * NOALLOC_HIST_BLOCKS;  // count, status
constexpr size_t NOALLOC_BYTES = OFF_WORDS + 256;

// about 3.9 MB: half-edge keys twice (sort ping-pong), flags, radix
// histograms and two words
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_mu;
void *g_base[64] = {};  // device address of g_noalloc_scratch, per device ordinal

}  // namespace

extern "C" hfcr_status hfcr_build_edges_noalloc(const int32_t *tris, int32_t n_tris, int32_t n_verts,
                                                int32_t *out, int64_t cap, int64_t *n_out,
                                                void *stream) {
    if (!n_out || n_tris < 0 || n_verts < 0 || (n_tris > 0 && (!tris || !out))) {
        hfcr::set_noctx_error("hfcr_build_edges_noalloc: bad arguments");
        return HFCR_ERR_ARG;
    }
    *n_out = 0;
    if (n_tris > NOALLOC_MAX_TRIS) {
        hfcr::set_noctx_error("hfcr_build_edges_noalloc: " + std::to_string(n_tris) +
                              " triangles exceed the fixed scratch limit of " +
                              std::to_string(NOALLOC_MAX_TRIS));
        return HFCR_ERR_CAPACITY;
    }
    if (cap < 3ll * n_tris) {
        hfcr::set_noctx_error("hfcr_build_edges_noalloc: cap must be at least 3 * n_tris");
        return HFCR_ERR_CAPACITY;
    }
    if (n_tris == 0) return HFCR_OK;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail("cudaGetDevice", ce);
    if (dev < 0 || dev >= 64) {
        hfcr::set_noctx_error("hfcr_build_edges_noalloc: device ordinal beyond 63");
        return HFCR_ERR_CUDA;
    }
    void *base = nullptr;
    {
        // the host-side name of a __device__ array is not a device address:
        // ask the runtime for this device's copy (once per device)
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_base[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return cuda_fail("cudaGetSymbolAddress", e);
            g_base[dev] = p;
        }
        base = g_base[dev];
    }
    char *b = (char *)base;
    cudaStream_t s = (cudaStream_t)stream;
    int *d_count = (int *)(b + OFF_WORDS);
    uint32_t *d_status = (uint32_t *)(b + OFF_WORDS + 4);
    hfcr::SortTemp t;
    t.hist = (unsigned *)(b + OFF_HIST);
    t.max_blocks = NOALLOC_HIST_BLOCKS;
    t.status = d_status;
    // the count and the status word carry over from the previous call
    if ((ce = cudaMemsetAsync(d_count, 0, 8, s)) != cudaSuccess)
        return cuda_fail("cudaMemsetAsync", ce);
    hfcr::build_edges(tris, n_tris, n_verts, out, d_count, (unsigned long long *)(b + OFF_KEYS),
                      (unsigned long long *)(b + OFF_KEYS_ALT), (unsigned *)(b + OFF_FLAGS), t,
                      d_status, s);
    // a launch error of this call's kernels, peeked rather than fetched: an
    // error state the caller's own earlier work left behind is not cleared
    // here (it is reported like a failure of this call)
    if ((ce = cudaPeekAtLastError()) != cudaSuccess) return cuda_fail("a kernel launch", ce);
    int words[2] = {0, 0};
    if ((ce = cudaMemcpyAsync(words, d_count, sizeof words, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail("cudaMemcpyAsync", ce);
    if ((ce = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail("cudaStreamSynchronize", ce);
    if (words[1] & hfcr::ST_BAD_INDEX) {
        hfcr::set_noctx_error("hfcr_build_edges_noalloc: a vertex index is out of range");
        return HFCR_ERR_ARG;
    }
    *n_out = words[0];
    return HFCR_OK;
}
