// Internal definitions shared by the fdcore translation units (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/fdcore.h"
#include "fd_jit_rt.cuh"
#include <vector>

// ---- error plumbing ---------------------------------------------------------
namespace fd {

fd_status set_error(fd_status st, const std::string &msg);
fd_status cuda_error(cudaError_t e, const char *what);

#define FD_CHECK_CUDA(call)                                     \
    do {                                                        \
        cudaError_t e__ = (call);                               \
        if (e__ != cudaSuccess) return ::fd::cuda_error(e__, #call); \
    } while (0)

#define FD_REQUIRE(cond, msg)                                   \
    do {                                                        \
        if (!(cond)) return ::fd::set_error(FD_EINVAL, (msg));  \
    } while (0)

// device-side status word (one per device, zero when healthy)
int *device_status_word();

// the sampler map's cos / sin table on the current device (filled on first use)
fd_status sc_table(const FdTab4 **out);

}  // namespace fd

// ---- tape format, version 4 (mirrors paper_2403_18840_gb300/fdgraph.py) ----------
enum : uint32_t {
    OP_FMA = 1,      // reserved (products and sums travel in bundles)
    OP_GLEAF = 2,    // G0 Taylor family from a momentum mask and two interaction lines
    OP_VLEAF = 3,    // V Taylor family from a momentum mask
    OP_RACC = 4,     // root accumulator += S[a] * exp(i pi x_line)
    OP_RFLUSH = 5,   // root d complete
    OP_CONST = 6,    // S[d] = f32 immediate
    OP_NOP = 7,      // padding
    OP_BUNDLE = 8,   // next n (1..8) words are independent FMAs, u16 (d, a, b, c) each
    OP_END = 63,
};

constexpr uint32_t TAPE_MAGIC = 0x50544446u;  // 'FDTP'
constexpr uint32_t TAPE_VERSION = 4;
constexpr int FD_CHUNK_WORDS = 1024;  // tape chunk staged in shared memory; bundles never straddle one
constexpr int FD_MAX_BUNDLE = 8;

struct TapeHeader {
    uint32_t magic, version, order, dim, n_roots, n_slots, n_instr, root_off, instr_off,
        total_bytes, n_mom, n_g, n_v, n_arith, r0, r1;
};


struct fd_graph {
    int device;
    int launch_threads = 0, launch_spt = 0;   // preferred CTA shape (0 = automatic)
    TapeHeader hdr;
    uint64_t *d_tape;            // device copy of the instruction words (16-byte aligned)
    uint32_t *d_roots;           // device root table: (n | m<<8 | l<<16 | dk<<24, re | im<<16)
    uint32_t h_roots[2 * 256];
    std::vector<uint64_t> h_tape;   // host copy of the validated instruction words
    // specialised straight-line kernel (fd_graph_jit), null until compiled
    cudaLibrary_t jit_lib = nullptr;
    cudaKernel_t jit_kernel = nullptr;
    int jit_threads = 0, jit_min_blocks = 0, jit_regs = 0, jit_local_bytes = 0, jit_modules = 0, jit_per_sm = 1;
    int jit_spt = 1;
    int jit_hist_cap = 0;           // floats of dynamic shared memory the kernel may take for a tile histogram
    int jit_sv_bytes = 0;           // dynamic shared memory of the per-sample inputs (before the histogram)
    float *jit_lc = nullptr;        // global leaf cache (lc_global): one region per resident CTA
    int64_t jit_lc_floats = 0;      // its size in floats
    double jit_compile_s = 0.0;
    bool jit_enabled = false;       // evaluation uses the specialised kernel
};

// validated host part of a graph (fd_api.cu)
fd_status graph_from_tape(const void *buf, size_t len, fd_graph &g);

// launches the specialised kernel of graph g for the instances in `args`
// (fd_jit.cu); the caller has reset the work counter
fd_status jit_launch(const fd_graph *g, EvalArgs &args, cudaStream_t stream);

struct fd_vegas {
    int device;
    int dim, n_bins;
    double *d_edges;   // [dim][n_bins+1]
    float *d_edges32;  // [dim][n_bins+1]
    double *d_hist;    // [dim][n_bins]
};

// ---- bounded mbarrier / bulk-copy helpers (inline PTX) ----------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared through the TMA engine, completing on `bar`.
// dst/src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar`; gives up after `limit` polls (returns false).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbarrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// status codes written to the device status word
constexpr int DEV_ST_TIMEOUT = 1;
