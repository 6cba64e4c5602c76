// C-ABI plumbing: errors, graph tapes, VEGAS maps, sample mapping and the
// host FP64 renormalisation post-process.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "fd_internal.cuh"

// ---- errors ----------------------------------------------------------------------
namespace fd {
static thread_local std::string g_last_error;

fd_status set_error(fd_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

fd_status cuda_error(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? FD_ENOMEM : FD_ECUDA;
}

int *device_status_word() {
    static std::mutex mu;
    static int *words[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!words[dev]) {
        int *p = nullptr;
        if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
        words[dev] = p;
    }
    return words[dev];
}
}  // namespace fd

extern "C" const char *fd_last_error(void) { return fd::g_last_error.c_str(); }

// Synchronise `stream` and report a device-side failure recorded by a kernel
// since the last call (bounded waits that gave up); clears the record.
extern "C" fd_status fd_device_status(void *stream) {
    FD_CHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int *w = fd::device_status_word();
    if (!w) return fd::set_error(FD_ECUDA, "no device status word");
    int h = 0;
    FD_CHECK_CUDA(cudaMemcpy(&h, w, sizeof(int), cudaMemcpyDeviceToHost));
    if (h == 0) return FD_OK;
    FD_CHECK_CUDA(cudaMemset(w, 0, sizeof(int)));
    return fd::set_error(FD_ETIMEOUT, "a kernel gave up waiting for a tape copy");
}

// ---- graphs ------------------------------------------------------------------------
fd_status validate_tape(const uint8_t *buf, size_t len, TapeHeader &h) {
    if (len < sizeof(TapeHeader)) return fd::set_error(FD_EFORMAT, "tape shorter than its header");
    memcpy(&h, buf, sizeof(TapeHeader));
    if (h.magic != TAPE_MAGIC) return fd::set_error(FD_EFORMAT, "bad tape magic");
    if (h.version != TAPE_VERSION) return fd::set_error(FD_EFORMAT, "unsupported tape version");
    if (h.order < 1 || h.order > (uint32_t)FD_MAX_ORDER) return fd::set_error(FD_EFORMAT, "order out of range");
    if (h.dim != 4 * h.order - 1) return fd::set_error(FD_EFORMAT, "dim != 4*order-1");
    if (h.n_roots < 1 || h.n_roots > 256) return fd::set_error(FD_EFORMAT, "root count out of range");
    if (h.n_slots < 2 || h.n_slots > 16383) return fd::set_error(FD_EFORMAT, "slot count out of range");
    if (h.n_instr < 1) return fd::set_error(FD_EFORMAT, "empty tape");
    if (h.total_bytes != len) return fd::set_error(FD_EFORMAT, "tape length differs from its header");
    if (h.root_off % 16 || h.instr_off % 16) return fd::set_error(FD_EFORMAT, "sections not 16-byte aligned");
    if ((uint64_t)h.root_off + 8ull * h.n_roots > len) return fd::set_error(FD_EFORMAT, "root table out of bounds");
    if ((uint64_t)h.instr_off + 8ull * h.n_instr > len) return fd::set_error(FD_EFORMAT, "instructions out of bounds");
    const uint32_t N = h.order;
    const uint32_t fixed = 2 + N;   // 0.0, 1.0, times of the N interaction lines
    const uint32_t S = h.n_slots;
    if (S < fixed) return fd::set_error(FD_EFORMAT, "slot count below the fixed slots");
    for (uint32_t r = 0; r < h.n_roots; ++r) {
        const uint8_t *p = buf + h.root_off + 8 * r;
        const uint32_t n = p[0], m = p[1], l = p[2], dk = p[3];
        if (n < 1 || n > N || n + m + l > N || dk > 1) return fd::set_error(FD_EFORMAT, "bad root (n, m, l, dk)");
    }
    std::vector<int> flushed(h.n_roots, 0);
    bool has_end = false;
    uint32_t in_bundle = 0;                 // FMA words still expected in the current bundle
    std::vector<uint32_t> bdst;             // destinations of the current bundle
    for (uint32_t k = 0; k < h.n_instr; ++k) {
        uint64_t w;
        memcpy(&w, buf + h.instr_off + 8ull * k, 8);
        if (in_bundle) {
            // bundle word: four u16 slot indices (d, a, b, c)
            const uint32_t d = (uint32_t)(w & 0xFFFFu), a = (uint32_t)((w >> 16) & 0xFFFFu),
                           b = (uint32_t)((w >> 32) & 0xFFFFu), c = (uint32_t)(w >> 48);
            bool ok = d >= fixed && d < S && a < S && b < S && c < S;
            for (uint32_t q : bdst) ok = ok && q != d;   // results may not share a slot
            bdst.push_back(d);
            if (!ok) return fd::set_error(FD_EFORMAT, "bundle word " + std::to_string(k) + " out of range");
            --in_bundle;
            continue;
        }
        const uint32_t op = (uint32_t)(w & 63u);
        const uint32_t d = (uint32_t)(w >> 6) & 16383u, a = (uint32_t)(w >> 20) & 16383u,
                       b = (uint32_t)(w >> 34) & 16383u, c = (uint32_t)(w >> 48) & 16383u;
        (void)c;
        bool ok = true;
        switch (op) {
            case OP_BUNDLE: {
                const uint32_t n = (uint32_t)(w >> 6) & 15u;
                ok = n >= 1 && n <= (uint32_t)FD_MAX_BUNDLE && k + n < h.n_instr &&
                     k / FD_CHUNK_WORDS == (k + n) / FD_CHUNK_WORDS;
                in_bundle = n;
                bdst.clear();
                break;
            }
            case OP_NOP: break;
            case OP_GLEAF:
            case OP_VLEAF: {
                const uint32_t la = (uint32_t)(w >> 34) & 7u, lb = (uint32_t)(w >> 37) & 7u;
                const uint32_t M = (uint32_t)(w >> 40) & 7u, dk = (uint32_t)(w >> 43) & 1u;
                const uint32_t width = (M + 1) * (dk ? 2 : 1);
                ok = d >= fixed && d + width <= S && M + dk <= (uint32_t)FD_MAX_M;
                for (uint32_t j = 0; j <= (uint32_t)FD_MAX_ORDER && ok; ++j) {
                    const uint32_t f = (a >> (2 * j)) & 3u;   // 0 absent, 1 plus, 3 minus
                    ok = f != 2u && (j <= N || f == 0u);
                }
                if (op == OP_GLEAF) ok = ok && la < N && lb < N;
                // above the d/dk flag: only a G leaf's FP64 flag
                ok = ok && (w >> (FD_LEAF_PRECISE_BIT + 1)) == 0 &&
                     (op == OP_GLEAF || ((w >> FD_LEAF_PRECISE_BIT) & 1u) == 0);
                break;
            }
            case OP_RACC: ok = a < S && b < N; break;
            case OP_RFLUSH:
                ok = d < h.n_roots;
                if (ok) ++flushed[d];
                break;
            case OP_CONST: ok = d >= fixed && d < S; break;
            case OP_END: has_end = (k == h.n_instr - 1); ok = has_end; break;
            default: ok = false;
        }
        if (!ok) return fd::set_error(FD_EFORMAT, "instruction " + std::to_string(k) + " (op " +
                                                      std::to_string(op) + ") out of range");
    }
    for (uint32_t r = 0; r < h.n_roots; ++r)
        if (flushed[r] != 1) return fd::set_error(FD_EFORMAT, "root " + std::to_string(r) + " not flushed exactly once");
    if (!has_end) return fd::set_error(FD_EFORMAT, "tape does not end with END");
    return FD_OK;
}

// Host part of a graph: validated header, instruction words and root table.
fd_status graph_from_tape(const void *buf, size_t len, fd_graph &g) {
    TapeHeader h;
    const fd_status st = validate_tape((const uint8_t *)buf, len, h);
    if (st != FD_OK) return st;
    g.hdr = h;
    g.h_tape.resize(h.n_instr);
    memcpy(g.h_tape.data(), (const uint8_t *)buf + h.instr_off, (size_t)h.n_instr * 8);
    for (uint32_t r = 0; r < h.n_roots; ++r) {
        const uint8_t *p = (const uint8_t *)buf + h.root_off + 8 * r;
        uint16_t re, im;
        memcpy(&re, p + 4, 2);
        memcpy(&im, p + 6, 2);
        g.h_roots[2 * r] = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
        g.h_roots[2 * r + 1] = (uint32_t)re | ((uint32_t)im << 16);
    }
    return FD_OK;
}

extern "C" fd_status fd_graph_load(const void *buf, size_t len, fd_graph **out) {
    FD_REQUIRE(buf && out, "buf and out are required");
    *out = nullptr;
    fd_graph *g = new fd_graph();
    const fd_status st = graph_from_tape(buf, len, *g);
    if (st != FD_OK) {
        delete g;
        return st;
    }
    const TapeHeader &h = g->hdr;
    cudaError_t e = cudaGetDevice(&g->device);
    const size_t ibytes = ((size_t)h.n_instr * 8 + 15) & ~(size_t)15;
    if (e == cudaSuccess) e = cudaMalloc(&g->d_tape, ibytes + 16);
    if (e == cudaSuccess) e = cudaMemset(g->d_tape, 0, ibytes + 16);
    if (e == cudaSuccess)
        e = cudaMemcpy(g->d_tape, g->h_tape.data(), (size_t)h.n_instr * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_roots, 8 * h.n_roots);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_roots, g->h_roots, 8 * h.n_roots, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(g->d_tape);
        cudaFree(g->d_roots);
        delete g;
        return fd::cuda_error(e, "graph upload");
    }
    // the sampler map's table on this device, filled here (before any stream
    // capture of an evaluation)
    const FdTab4 *tab = nullptr;
    const fd_status ts = fd::sc_table(&tab);
    if (ts != FD_OK) {
        cudaFree(g->d_tape);
        cudaFree(g->d_roots);
        delete g;
        return ts;
    }
    *out = g;
    return FD_OK;
}

extern "C" fd_status fd_graph_info(const fd_graph *g, int32_t *n_roots, int32_t *dim, int64_t *n_instr,
                                   int32_t *n_slots) {
    FD_REQUIRE(g, "null graph");
    if (n_roots) *n_roots = (int32_t)g->hdr.n_roots;
    if (dim) *dim = (int32_t)g->hdr.dim;
    if (n_instr) *n_instr = (int64_t)g->hdr.n_instr;
    if (n_slots) *n_slots = (int32_t)g->hdr.n_slots;
    return FD_OK;
}

extern "C" fd_status fd_graph_roots(const fd_graph *g, int32_t *roots) {
    FD_REQUIRE(g && roots, "graph and roots are required");
    for (uint32_t r = 0; r < g->hdr.n_roots; ++r) {
        const uint32_t t = g->h_roots[2 * r];
        roots[4 * r] = (int32_t)(t & 255u);
        roots[4 * r + 1] = (int32_t)((t >> 8) & 255u);
        roots[4 * r + 2] = (int32_t)((t >> 16) & 255u);
        roots[4 * r + 3] = (int32_t)((t >> 24) & 255u);
    }
    return FD_OK;
}

extern "C" void fd_graph_free(fd_graph *g) {
    if (!g) return;
    if (g->jit_lib) cudaLibraryUnload(g->jit_lib);
    if (g->jit_lc) cudaFree(g->jit_lc);
    cudaFree(g->d_tape);
    cudaFree(g->d_roots);
    delete g;
}

// ---- VEGAS ---------------------------------------------------------------------------
namespace {
__global__ void edges_to_f32(const double *e, float *e32, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) e32[i] = (float)e[i];
}

// One CTA per dimension (Lepage's grid refinement, FP64).
__global__ void vegas_update_kernel(double *edges, float *edges32, double *hist, int nb, double alpha) {
    extern __shared__ double sh[];
    double *d = sh;              // [nb] histogram
    double *r = sh + nb;         // [nb] damped importance, then inclusive scan
    double *e = sh + 2 * nb;     // [nb+1] old edges
    double *red = sh + 3 * nb + 1;  // [blockDim] reduction scratch
    const int dim = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
    double *E = edges + (size_t)dim * (nb + 1);
    double *H = hist + (size_t)dim * nb;
    for (int i = tid; i < nb; i += T) d[i] = H[i];
    for (int i = tid; i <= nb; i += T) e[i] = E[i];
    __syncthreads();
    // smoothing: 3-point average, 2-point at the ends
    for (int i = tid; i < nb; i += T) {
        double s;
        if (nb == 1) s = d[0];
        else if (i == 0) s = (d[0] + d[1]) / 2.0;
        else if (i == nb - 1) s = (d[nb - 2] + d[nb - 1]) / 2.0;
        else s = (d[i - 1] + d[i] + d[i + 1]) / 3.0;
        r[i] = s;
    }
    __syncthreads();
    // total (fixed-order: per-thread strided sums, then a tree)
    double part = 0.0;
    for (int i = tid; i < nb; i += T) part += r[i];
    red[tid] = part;
    __syncthreads();
    for (int s = T / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] += red[tid + s];
        __syncthreads();
    }
    const double S = red[0];
    __syncthreads();
    if (!(S > 0.0)) {
        for (int i = tid; i < nb; i += T) H[i] = 0.0;
        return;
    }
    for (int i = tid; i < nb; i += T) {
        const double rho = r[i] / S;
        double v;
        if (rho <= 0.0) v = 0.0;
        else if (rho >= 1.0) v = 1.0;
        else v = pow((rho - 1.0) / log(rho), alpha);
        r[i] = v;
    }
    __syncthreads();
    // inclusive scan of r (sequential in thread 0: nb <= a few thousand)
    if (tid == 0) {
        double acc = 0.0;
        for (int i = 0; i < nb; ++i) {
            acc += r[i];
            d[i] = acc;     // d now holds the inclusive scan
        }
    }
    __syncthreads();
    const double R = d[nb - 1];
    if (!(R > 0.0)) {
        for (int i = tid; i < nb; i += T) H[i] = 0.0;
        return;
    }
    const double target = R / nb;
    for (int t = tid + 1; t < nb; t += T) {
        const double want = t * target;
        // first bin j with inclusive cumulative >= want (j <= nb-1)
        int lo = 0, hi = nb - 1;
        while (lo < hi) {
            const int mid = (lo + hi) / 2;
            if (d[mid] >= want) hi = mid;
            else lo = mid + 1;
        }
        const int j = lo;
        const double before = j ? d[j - 1] : 0.0;
        const double rj = r[j];
        double frac = rj > 0.0 ? (want - before) / rj : 0.0;
        frac = fmin(fmax(frac, 0.0), 1.0);
        E[t] = e[j] + frac * (e[j + 1] - e[j]);
    }
    if (tid == 0) {
        E[0] = 0.0;
        E[nb] = 1.0;
    }
    __syncthreads();
    for (int i = tid; i <= nb; i += T) edges32[(size_t)dim * (nb + 1) + i] = (float)E[i];
    for (int i = tid; i < nb; i += T) H[i] = 0.0;
}

struct MapRef {
    double *edges;
    float *edges32;
    double *hist;
    int dim;
};
struct BatchMaps {
    MapRef m[256];
};

// Batched update: block (dim, map); same algorithm as vegas_update_kernel.
__global__ void vegas_update_batch_kernel(const __grid_constant__ BatchMaps B, int nb, double alpha) {
    const MapRef M = B.m[blockIdx.y];
    if ((int)blockIdx.x >= M.dim) return;
    extern __shared__ double sh[];
    double *d = sh;
    double *r = sh + nb;
    double *e = sh + 2 * nb;
    double *red = sh + 3 * nb + 1;
    const int dim = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
    double *E = M.edges + (size_t)dim * (nb + 1);
    double *H = M.hist + (size_t)dim * nb;
    for (int i = tid; i < nb; i += T) d[i] = H[i];
    for (int i = tid; i <= nb; i += T) e[i] = E[i];
    __syncthreads();
    for (int i = tid; i < nb; i += T) {
        double s;
        if (nb == 1) s = d[0];
        else if (i == 0) s = (d[0] + d[1]) / 2.0;
        else if (i == nb - 1) s = (d[nb - 2] + d[nb - 1]) / 2.0;
        else s = (d[i - 1] + d[i] + d[i + 1]) / 3.0;
        r[i] = s;
    }
    __syncthreads();
    double part = 0.0;
    for (int i = tid; i < nb; i += T) part += r[i];
    red[tid] = part;
    __syncthreads();
    for (int s2 = T / 2; s2 > 0; s2 >>= 1) {
        if (tid < s2) red[tid] += red[tid + s2];
        __syncthreads();
    }
    const double S = red[0];
    __syncthreads();
    if (!(S > 0.0)) {
        for (int i = tid; i < nb; i += T) H[i] = 0.0;
        return;
    }
    for (int i = tid; i < nb; i += T) {
        const double rho = r[i] / S;
        r[i] = rho <= 0.0 ? 0.0 : (rho >= 1.0 ? 1.0 : pow((rho - 1.0) / log(rho), alpha));
    }
    __syncthreads();
    if (tid == 0) {
        double acc = 0.0;
        for (int i = 0; i < nb; ++i) {
            acc += r[i];
            d[i] = acc;
        }
    }
    __syncthreads();
    const double R = d[nb - 1];
    if (!(R > 0.0)) {
        for (int i = tid; i < nb; i += T) H[i] = 0.0;
        return;
    }
    const double target = R / nb;
    for (int t = tid + 1; t < nb; t += T) {
        const double want = t * target;
        int lo = 0, hi = nb - 1;
        while (lo < hi) {
            const int mid = (lo + hi) / 2;
            if (d[mid] >= want) hi = mid;
            else lo = mid + 1;
        }
        const int j = lo;
        const double before = j ? d[j - 1] : 0.0;
        const double rj = r[j];
        double frac = rj > 0.0 ? (want - before) / rj : 0.0;
        frac = fmin(fmax(frac, 0.0), 1.0);
        E[t] = e[j] + frac * (e[j + 1] - e[j]);
    }
    if (tid == 0) {
        E[0] = 0.0;
        E[nb] = 1.0;
    }
    __syncthreads();
    for (int i = tid; i <= nb; i += T) M.edges32[(size_t)dim * (nb + 1) + i] = (float)E[i];
    for (int i = tid; i < nb; i += T) H[i] = 0.0;
}

__global__ void map_samples_kernel(const float *edges32, int nb, uint32_t seed_lo, uint32_t seed_hi,
                                   uint32_t iter, uint32_t inst, int64_t n, int dim, float *x, float *w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t c0 = (uint32_t)(uint64_t)i, c1 = (uint32_t)((uint64_t)i >> 32);
    float jac = 1.0f;
    for (int blk = 0; 4 * blk < dim; ++blk) {
        const u32x4 r = philox4x32_10(u32x4{c0, c1, iter, (inst << 8) | (uint32_t)blk}, seed_lo, seed_hi);
        const uint32_t wv[4] = {r.x, r.y, r.z, r.w};
        for (int q = 0; q < 4 && 4 * blk + q < dim; ++q) {
            const int d = 4 * blk + q;
            float u = word_to_uniform(wv[q]);
            if (edges32) {
                const float y = u * (float)nb;
                const int bin = min((int)y, nb - 1);
                const float *e = edges32 + (int64_t)d * (nb + 1);
                const float lo = e[bin], hi = e[bin + 1];
                u = fmaf(y - (float)bin, hi - lo, lo);
                jac *= (float)nb * (hi - lo);
            }
            x[(int64_t)d * n + i] = u;
        }
    }
    if (w) w[i] = jac;
}
}  // namespace

extern "C" fd_status fd_vegas_create(int32_t dim, int32_t n_bins, fd_vegas **out) {
    FD_REQUIRE(out, "out is required");
    *out = nullptr;
    FD_REQUIRE(dim >= 1 && dim <= FD_MAX_DIM, "dim out of range");
    FD_REQUIRE(n_bins >= 1 && n_bins <= 8192, "n_bins out of range");
    fd_vegas *m = new fd_vegas();
    m->dim = dim;
    m->n_bins = n_bins;
    FD_CHECK_CUDA(cudaGetDevice(&m->device));
    const size_t ne = (size_t)dim * (n_bins + 1);
    std::vector<double> e(ne);
    for (int d = 0; d < dim; ++d)
        for (int i = 0; i <= n_bins; ++i) e[(size_t)d * (n_bins + 1) + i] = (double)i / n_bins;
    cudaError_t err = cudaMalloc(&m->d_edges, ne * 8);
    if (err == cudaSuccess) err = cudaMalloc(&m->d_edges32, ne * 4);
    if (err == cudaSuccess) err = cudaMalloc(&m->d_hist, (size_t)dim * n_bins * 8);
    if (err == cudaSuccess) err = cudaMemset(m->d_hist, 0, (size_t)dim * n_bins * 8);
    if (err != cudaSuccess) {
        fd_vegas_free(m);
        return fd::cuda_error(err, "fd_vegas_create");
    }
    fd_status st = fd_vegas_set_edges(m, e.data());
    if (st != FD_OK) {
        fd_vegas_free(m);
        return st;
    }
    *out = m;
    return FD_OK;
}

extern "C" void fd_vegas_free(fd_vegas *m) {
    if (!m) return;
    cudaFree(m->d_edges);
    cudaFree(m->d_edges32);
    cudaFree(m->d_hist);
    delete m;
}

extern "C" fd_status fd_vegas_set_edges(fd_vegas *m, const double *edges) {
    FD_REQUIRE(m && edges, "map and edges are required");
    const int nb = m->n_bins;
    for (int d = 0; d < m->dim; ++d) {
        const double *e = edges + (size_t)d * (nb + 1);
        FD_REQUIRE(e[0] == 0.0 && e[nb] == 1.0, "edges must start at 0 and end at 1");
        for (int i = 0; i < nb; ++i) FD_REQUIRE(e[i + 1] > e[i], "edges must be strictly increasing");
    }
    const size_t ne = (size_t)m->dim * (nb + 1);
    FD_CHECK_CUDA(cudaMemcpy(m->d_edges, edges, ne * 8, cudaMemcpyHostToDevice));
    edges_to_f32<<<(int)((ne + 255) / 256), 256>>>(m->d_edges, m->d_edges32, (int)ne);
    FD_CHECK_CUDA(cudaGetLastError());
    FD_CHECK_CUDA(cudaDeviceSynchronize());
    return FD_OK;
}

extern "C" fd_status fd_vegas_get_edges(const fd_vegas *m, double *edges) {
    FD_REQUIRE(m && edges, "map and edges are required");
    FD_CHECK_CUDA(cudaDeviceSynchronize());
    FD_CHECK_CUDA(cudaMemcpy(edges, m->d_edges, (size_t)m->dim * (m->n_bins + 1) * 8, cudaMemcpyDeviceToHost));
    return FD_OK;
}

extern "C" fd_status fd_vegas_get_hist(const fd_vegas *m, double *hist) {
    FD_REQUIRE(m && hist, "map and hist are required");
    FD_CHECK_CUDA(cudaDeviceSynchronize());
    FD_CHECK_CUDA(cudaMemcpy(hist, m->d_hist, (size_t)m->dim * m->n_bins * 8, cudaMemcpyDeviceToHost));
    return FD_OK;
}

extern "C" fd_status fd_vegas_set_hist(fd_vegas *m, const double *hist) {
    FD_REQUIRE(m && hist, "map and hist are required");
    for (size_t k = 0; k < (size_t)m->dim * m->n_bins; ++k)
        FD_REQUIRE(hist[k] >= 0.0 && std::isfinite(hist[k]), "histogram entries must be finite and >= 0");
    FD_CHECK_CUDA(cudaDeviceSynchronize());
    FD_CHECK_CUDA(cudaMemcpy(m->d_hist, hist, (size_t)m->dim * m->n_bins * 8, cudaMemcpyHostToDevice));
    return FD_OK;
}

extern "C" fd_status fd_vegas_clear_hist(fd_vegas *m, void *stream) {
    FD_REQUIRE(m, "map is required");
    FD_CHECK_CUDA(cudaMemsetAsync(m->d_hist, 0, (size_t)m->dim * m->n_bins * 8, (cudaStream_t)stream));
    return FD_OK;
}

extern "C" fd_status fd_vegas_update(fd_vegas *m, double alpha, void *stream) {
    FD_REQUIRE(m, "map is required");
    FD_REQUIRE(alpha >= 0.0 && alpha <= 4.0 && std::isfinite(alpha), "alpha out of range");
    const int nb = m->n_bins, T = 256;
    const size_t sh = (size_t)(3 * nb + 1 + T) * 8;
    FD_REQUIRE(sh <= 227 * 1024, "too many bins for the update kernel");
    if (sh > 48 * 1024)
        FD_CHECK_CUDA(cudaFuncSetAttribute(vegas_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    vegas_update_kernel<<<m->dim, T, sh, (cudaStream_t)stream>>>(m->d_edges, m->d_edges32, m->d_hist, nb, alpha);
    FD_CHECK_CUDA(cudaGetLastError());
    return FD_OK;
}

extern "C" fd_status fd_vegas_update_batch(fd_vegas *const *maps, int32_t n_maps, double alpha, void *stream) {
    FD_REQUIRE(maps && n_maps >= 1 && n_maps <= 256, "1..256 maps are required");
    FD_REQUIRE(alpha >= 0.0 && alpha <= 4.0 && std::isfinite(alpha), "alpha out of range");
    static thread_local BatchMaps B;   // kernel argument (copied at launch); per host thread
    int nb = -1, dmax = 0;
    for (int k = 0; k < n_maps; ++k) {
        FD_REQUIRE(maps[k], "null map");
        if (nb < 0) nb = maps[k]->n_bins;
        FD_REQUIRE(maps[k]->n_bins == nb, "all maps of a batched update need the same bin count");
        B.m[k] = MapRef{maps[k]->d_edges, maps[k]->d_edges32, maps[k]->d_hist, maps[k]->dim};
        dmax = std::max(dmax, maps[k]->dim);
    }
    const int T = 256;
    const size_t sh = (size_t)(3 * nb + 1 + T) * 8;
    FD_REQUIRE(sh <= 227 * 1024, "too many bins for the update kernel");
    if (sh > 48 * 1024)
        FD_CHECK_CUDA(cudaFuncSetAttribute(vegas_update_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    vegas_update_batch_kernel<<<dim3(dmax, n_maps), T, sh, (cudaStream_t)stream>>>(B, nb, alpha);
    FD_CHECK_CUDA(cudaGetLastError());
    return FD_OK;
}

extern "C" fd_status fd_map_samples(const fd_vegas *map, uint64_t seed, uint64_t iter, int32_t inst, int64_t n,
                                    int32_t dim, float *x, float *w, void *stream) {
    FD_REQUIRE(x, "x is required");
    FD_REQUIRE(n > 0 && dim >= 1 && dim <= FD_MAX_DIM, "bad n or dim");
    FD_REQUIRE(inst >= 0 && inst < (1 << 24), "instance index out of range");
    if (map) FD_REQUIRE(map->dim == dim, "map dimension differs");
    const int T = 256;
    map_samples_kernel<<<(unsigned)((n + T - 1) / T), T, 0, (cudaStream_t)stream>>>(
        map ? map->d_edges32 : nullptr, map ? map->n_bins : 1, (uint32_t)seed, (uint32_t)(seed >> 32),
        (uint32_t)iter, (uint32_t)inst, n, dim, x, w);
    FD_CHECK_CUDA(cudaGetLastError());
    return FD_OK;
}

// ---- post-processing (host FP64) ------------------------------------------------------
namespace {
using Series = std::vector<double>;

Series mul(const Series &a, const Series &b, int N) {
    Series o(N + 1, 0.0);
    for (int i = 0; i <= N; ++i)
        for (int j = 0; i + j <= N; ++j) o[i + j] += a[i] * b[j];
    return o;
}

// sum_{n,m,l} xi^(n+l) dmu(xi)^m/m! (-Lambda)^l/l! c[n][m][l] as a xi-series
Series substitute(const double *c, const Series &dmu, double Lam, int N, int Nc) {
    Series out(N + 1, 0.0);
    std::vector<Series> powers(N + 1);
    powers[0] = Series(N + 1, 0.0);
    powers[0][0] = 1.0;
    for (int m = 1; m <= N; ++m) powers[m] = mul(powers[m - 1], dmu, N);
    for (int n = 1; n <= N; ++n)
        for (int m = 0; n + m <= N; ++m)
            for (int l = 0; n + m + l <= N; ++l) {
                const double v = c[((size_t)n * (Nc + 1) + m) * (Nc + 1) + l];
                if (v == 0.0 || n + l > N) continue;
                double f = v * std::pow(-Lam, l);
                for (int q = 2; q <= l; ++q) f /= q;
                for (int q = 2; q <= m; ++q) f /= q;
                for (int k = 0; n + l + k <= N; ++k) out[n + l + k] += f * powers[m][k];
            }
    return out;
}
}  // namespace

extern "C" fd_status fd_postprocess(int32_t N, const double *sigma_re, const double *sigma_im,
                                    const double *dsigma_re, double k_F, double beta, double Lambda, double *dmu_out,
                                    double *a_out, double *b_out, double *meff_out) {
    FD_REQUIRE(N >= 1 && N <= 12, "N out of range");
    FD_REQUIRE(sigma_re && sigma_im && dsigma_re, "inputs are required");
    FD_REQUIRE(k_F > 0 && beta > 0 && std::isfinite(Lambda), "bad k_F, beta or Lambda");
    const double w0 = M_PI / beta;
    Series dmu(N + 1, 0.0);
    for (int order = 1; order <= N; ++order) {
        Series s = substitute(sigma_re, dmu, Lambda, order, N);
        dmu[order] = s[order];
    }
    const size_t cnt = (size_t)(N + 1) * (N + 1) * (N + 1);
    std::vector<double> ac(cnt), bc(cnt);
    for (size_t k = 0; k < cnt; ++k) {
        ac[k] = dsigma_re[k] / (2.0 * k_F);
        bc[k] = sigma_im[k] / w0;
    }
    Series a = substitute(ac.data(), dmu, Lambda, N, N);
    Series b = substitute(bc.data(), dmu, Lambda, N, N);
    Series onea = a, oneb(N + 1);
    onea[0] += 1.0;
    for (int i = 0; i <= N; ++i) oneb[i] = -b[i];
    oneb[0] += 1.0;
    Series c(N + 1, 0.0);
    for (int i = 0; i <= N; ++i) {
        double s = oneb[i];
        for (int j = 0; j < i; ++j) s -= c[j] * onea[i - j];
        c[i] = s / onea[0];
    }
    double acc = 0.0;
    for (int i = 0; i <= N; ++i) {
        acc += c[i];
        if (dmu_out) dmu_out[i] = dmu[i];
        if (a_out) a_out[i] = a[i];
        if (b_out) b_out[i] = b[i];
        if (meff_out) meff_out[i] = acc;
    }
    return FD_OK;
}

// ---- throughput probes (FP32 FMA, SFU ex2 / rcp) ------------------------------------
namespace {
// 8 independent dependency chains per thread so the pipe, not latency, bounds the rate
template <int KIND>
__global__ void peak_kernel(float *out, int iters, float seed) {
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = seed + 0.001f * (threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (KIND == 0) {
                v[j] = fmaf(v[j], 0.9999999f, 1e-7f);
            } else if (KIND == 1) {
                float r;
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v[j]));
                v[j] = r * -0.5f;
            } else {
                float r;
                asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v[j]));
                v[j] = r + 1.0f;   // continued fraction: nothing to fold
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += v[j];
    if (s == 12345.678f) out[threadIdx.x] = s;   // keeps the work alive
}

// packed FP32: 8 independent chains of two-lane FMAs (one instruction, 4 flops)
__global__ void peak_kernel_f32x2(float *out, int iters, float seed) {
    float2 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = make_float2(seed + 0.001f * (threadIdx.x + j), seed - 0.001f * j);
    const float2 a = make_float2(0.9999999f, 0.9999998f), c = make_float2(1e-7f, 2e-7f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = __ffma2_rn(v[j], a, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += v[j].x + v[j].y;
    if (s == 12345.678f) out[threadIdx.x] = s;
}
}  // namespace

// Measured throughput of one pipe on the current device (synchronous):
// kind 0 = FP32 FMA (flops, FMA = 2), 1 = SFU ex2, 2 = SFU rcp (results),
// 3 = packed two-lane FP32 FMA (flops, 4 per instruction).
extern "C" fd_status fd_measure_peak(int32_t kind, double *ops_per_s) {
    FD_REQUIRE(ops_per_s && kind >= 0 && kind <= 3, "kind in 0..3 and an output are required");
    int dev = 0, n_sm = 0;
    FD_CHECK_CUDA(cudaGetDevice(&dev));
    FD_CHECK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    float *out = nullptr;
    FD_CHECK_CUDA(cudaMalloc(&out, 1024 * sizeof(float)));
    const int threads = 512, blocks = n_sm * 4, iters = (kind == 0 || kind == 3) ? 8192 : 2048;
    cudaEvent_t a, b;
    FD_CHECK_CUDA(cudaEventCreate(&a));
    FD_CHECK_CUDA(cudaEventCreate(&b));
    auto launch = [&]() {
        if (kind == 0) peak_kernel<0><<<blocks, threads>>>(out, iters, 1.0f);
        else if (kind == 1) peak_kernel<1><<<blocks, threads>>>(out, iters, 0.5f);
        else if (kind == 2) peak_kernel<2><<<blocks, threads>>>(out, iters, 1.5f);
        else peak_kernel_f32x2<<<blocks, threads>>>(out, iters, 1.0f);
    };
    launch();
    FD_CHECK_CUDA(cudaGetLastError());
    FD_CHECK_CUDA(cudaEventRecord(a));
    for (int r = 0; r < 5; ++r) launch();
    FD_CHECK_CUDA(cudaEventRecord(b));
    FD_CHECK_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    FD_CHECK_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    const double ops = 5.0 * blocks * threads * (double)iters * 8.0 * (kind == 0 ? 2.0 : kind == 3 ? 4.0 : 1.0);
    *ops_per_s = ops / (ms * 1e-3);
    return FD_OK;
}
