// Specialised integrand kernels: the validated instruction tape of a graph is
// translated into straight-line CUDA and compiled at run time for the device
// (NVRTC, then nvJitLink when the code is split into several modules).
//
// Why: the tape interpreter keeps every intermediate value of a sample in
// shared memory, so each FMA costs three shared loads and one store and the
// interpreter is bound by shared-memory bandwidth far below the FP32 pipe.
// In straight-line code the intermediates live in registers and the FP32 and
// SFU pipes become the bound.  The paper compiles its graphs to code for the
// same reason (Sec. VI.A: the graphs are compiled once and evaluated in
// batches); here the compilation starts from the same tape the interpreter
// runs, so both paths evaluate the same contraction.
//
// Translation.  The contraction of a root is a sum over root-accumulate
// instructions (RACC: value x exp(i pi x_line)); the backward slice of each
// RACC through the tape's slot definitions is one straight-line device
// function (its leaves included).  Slices are written in SSA form (every
// definition a new name, bundles read their operands before writing).  Small
// graphs go into one module with the slices inlined (the compiler then shares
// leaves between slices); large graphs are split into modules of similar size
// that compile in parallel, with the slices as separate functions linked into
// the kernel module.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <unistd.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "fd_internal.cuh"

namespace {

const char kRuntimeHeader[] =
#include "fd_jit_rt.inc"
    ;

constexpr int kJitVersion = 4;              // bump when the generated code changes meaning
constexpr double kSingleModuleCost = 3500;  // below this the graph compiles as one module

// ---- run-time compiler entry points (resolved with dlopen on first use) ---------
typedef int (*nvrtcCreateProgram_t)(void **, const char *, const char *, int, const char *const *,
                                    const char *const *);
typedef int (*nvrtcCompileProgram_t)(void *, int, const char *const *);
typedef int (*nvrtcGetSize_t)(void *, size_t *);
typedef int (*nvrtcGetData_t)(void *, char *);
typedef int (*nvrtcDestroyProgram_t)(void **);
typedef int (*njlCreate_t)(void **, uint32_t, const char **);
typedef int (*njlDestroy_t)(void **);
typedef int (*njlAddData_t)(void *, int, const void *, size_t, const char *);
typedef int (*njlComplete_t)(void *);
typedef int (*njlGetSize_t)(void *, size_t *);
typedef int (*njlGetData_t)(void *, void *);
typedef int (*njlGetLog_t)(void *, char *);

struct Rtc {
    bool ok = false;
    std::string why;
    nvrtcCreateProgram_t create;
    nvrtcCompileProgram_t compile;
    nvrtcGetSize_t log_size, cubin_size;
    nvrtcGetData_t log, cubin;
    nvrtcDestroyProgram_t destroy;
    njlCreate_t l_create;
    njlDestroy_t l_destroy;
    njlAddData_t l_add;
    njlComplete_t l_complete;
    njlGetSize_t l_cubin_size, l_log_size;
    njlGetData_t l_cubin;
    njlGetLog_t l_log;
};

#ifndef FD_CUDA_LIBDIR
#define FD_CUDA_LIBDIR ""
#endif

void *open_lib(const char *name) {
    void *h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
    if (!h && FD_CUDA_LIBDIR[0]) {
        const std::string p = std::string(FD_CUDA_LIBDIR) + "/" + name;
        h = dlopen(p.c_str(), RTLD_NOW | RTLD_LOCAL);
    }
    return h;
}

const Rtc &rtc() {
    static Rtc R;
    static std::once_flag once;
    std::call_once(once, [] {
        void *a = open_lib("libnvrtc.so.13");
        void *b = open_lib("libnvJitLink.so.13");
        if (!a || !b) {
            R.why = "libnvrtc.so.13 / libnvJitLink.so.13 not found";
            return;
        }
        bool ok = true;
        auto sym = [&](void *h, const char *n) {
            void *p = dlsym(h, n);
            if (!p) ok = false;
            return p;
        };
        R.create = (nvrtcCreateProgram_t)sym(a, "nvrtcCreateProgram");
        R.compile = (nvrtcCompileProgram_t)sym(a, "nvrtcCompileProgram");
        R.log_size = (nvrtcGetSize_t)sym(a, "nvrtcGetProgramLogSize");
        R.log = (nvrtcGetData_t)sym(a, "nvrtcGetProgramLog");
        R.cubin_size = (nvrtcGetSize_t)sym(a, "nvrtcGetCUBINSize");
        R.cubin = (nvrtcGetData_t)sym(a, "nvrtcGetCUBIN");
        R.destroy = (nvrtcDestroyProgram_t)sym(a, "nvrtcDestroyProgram");
        R.l_create = (njlCreate_t)sym(b, "__nvJitLinkCreate_13_0");
        R.l_destroy = (njlDestroy_t)sym(b, "__nvJitLinkDestroy_13_0");
        R.l_add = (njlAddData_t)sym(b, "__nvJitLinkAddData_13_0");
        R.l_complete = (njlComplete_t)sym(b, "__nvJitLinkComplete_13_0");
        R.l_cubin_size = (njlGetSize_t)sym(b, "__nvJitLinkGetLinkedCubinSize_13_0");
        R.l_cubin = (njlGetData_t)sym(b, "__nvJitLinkGetLinkedCubin_13_0");
        R.l_log_size = (njlGetSize_t)sym(b, "__nvJitLinkGetErrorLogSize_13_0");
        R.l_log = (njlGetLog_t)sym(b, "__nvJitLinkGetErrorLog_13_0");
        R.ok = ok;
        if (!ok) R.why = "run-time compiler symbols missing";
    });
    return R;
}

// ---- tape decoding and slicing ---------------------------------------------------
struct TIns {
    uint32_t op;
    uint32_t w;      // index of the instruction word
    uint32_t n;      // bundle: member count (members at w + 1 .. w + n)
};

struct Slice {
    uint32_t racc;                                // index into the instruction list
    int root, line;
    std::vector<std::pair<uint32_t, uint32_t>> keep;   // (instruction, kept bundle members bitmask)
    int n_fma = 0, n_leaf = 0;
    double cost() const { return n_fma + 30.0 * n_leaf; }
};

inline uint32_t fa(uint64_t w) { return (uint32_t)(w >> 20) & 16383u; }
inline uint32_t fd_(uint64_t w) { return (uint32_t)(w >> 6) & 16383u; }

int leaf_outputs(uint64_t w) {
    const int M = (int)((w >> 40) & 7u), dk = (int)((w >> 43) & 1u);
    return (M + 1) * (1 + dk);
}

std::vector<TIns> decode(const std::vector<uint64_t> &words) {
    std::vector<TIns> out;
    for (uint32_t k = 0; k < words.size(); ++k) {
        const uint64_t w = words[k];
        const uint32_t op = (uint32_t)(w & 63u);
        if (op == OP_BUNDLE) {
            const uint32_t n = (uint32_t)(w >> 6) & 15u;
            out.push_back({op, k, n});
            k += n;
            continue;
        }
        if (op == OP_NOP) continue;
        out.push_back({op, k, 0});
        if (op == OP_END) break;
    }
    return out;
}

std::vector<Slice> make_slices(const std::vector<TIns> &ins, const std::vector<uint64_t> &words, int n_slots) {
    std::vector<Slice> out;
    std::vector<char> need(n_slots + 1, 0);
    // root of each RACC: the next RFLUSH names it
    std::vector<int> root_of(ins.size(), -1);
    int cur = -1;
    for (int i = (int)ins.size() - 1; i >= 0; --i) {
        if (ins[i].op == OP_RFLUSH) cur = (int)fd_(words[ins[i].w]);
        root_of[i] = cur;
    }
    for (uint32_t i = 0; i < ins.size(); ++i) {
        if (ins[i].op != OP_RACC) continue;
        Slice s;
        s.racc = i;
        s.root = root_of[i];
        s.line = (int)((words[ins[i].w] >> 34) & 7u);
        std::fill(need.begin(), need.end(), 0);
        need[fa(words[ins[i].w])] = 1;
        for (int j = (int)i - 1; j >= 0; --j) {
            const TIns &t = ins[j];
            if (t.op == OP_BUNDLE) {
                uint32_t mask = 0;
                for (uint32_t q = 0; q < t.n; ++q)
                    if (need[words[t.w + 1 + q] & 0xFFFFu]) mask |= 1u << q;
                if (!mask) continue;
                for (uint32_t q = 0; q < t.n; ++q)
                    if (mask >> q & 1u) need[words[t.w + 1 + q] & 0xFFFFu] = 0;
                for (uint32_t q = 0; q < t.n; ++q) {
                    if (!(mask >> q & 1u)) continue;
                    const uint64_t m = words[t.w + 1 + q];
                    need[(m >> 16) & 0xFFFFu] = 1;
                    need[(m >> 32) & 0xFFFFu] = 1;
                    need[(m >> 48) & 0xFFFFu] = 1;
                    ++s.n_fma;
                }
                s.keep.push_back({(uint32_t)j, mask});
            } else if (t.op == OP_GLEAF || t.op == OP_VLEAF) {
                const uint64_t w = words[t.w];
                const uint32_t d = fd_(w);
                const int no = leaf_outputs(w);
                bool any = false;
                for (int q = 0; q < no; ++q) any = any || need[d + q];
                if (!any) continue;
                for (int q = 0; q < no; ++q) need[d + q] = 0;
                s.keep.push_back({(uint32_t)j, 0});
                ++s.n_leaf;
            } else if (t.op == OP_CONST) {
                const uint32_t d = fd_(words[t.w]);
                if (!need[d]) continue;
                need[d] = 0;
                s.keep.push_back({(uint32_t)j, 0});
            }
        }
        std::reverse(s.keep.begin(), s.keep.end());
        out.push_back(std::move(s));
    }
    return out;
}

// ---- source emission ---------------------------------------------------------------
std::string fnum(float f) {
    uint32_t b;
    memcpy(&b, &f, 4);
    char buf[48];
    snprintf(buf, sizeof buf, "__int_as_float(0x%08xu)", b);
    return buf;
}

// signed momentum sums of a 2-bit-per-variable mask: grid parts (x, y, z),
// remainders (xl, yl, zl) and the k_ext coefficient.  cast: a prefix for the
// remainder terms.
struct MomExpr {
    std::string x, y, z, xl, yl, zl, ks;
};

MomExpr momentum_expr(uint32_t mask, int N, const std::string &cast = "") {
    auto coef = [&](int j) { return (int)(((int32_t)(mask << (30 - 2 * j))) >> 30); };
    // -a + b is written b - a (the same value bit for bit, and one operation
    // fewer in the packed code); the order of the later terms is kept
    auto sum = [&](const char *comp, const char *ext, const std::string &pre) {
        std::vector<std::pair<int, std::string>> terms;
        if (ext && coef(0)) terms.push_back({coef(0), pre + ext});
        for (int j = 1; j <= N; ++j)
            if (coef(j)) terms.push_back({coef(j), pre + "V." + comp + "[" + std::to_string(j - 1) + "]"});
        if (terms.empty()) return std::string("0.0f");
        if (terms.size() >= 2 && terms[0].first < 0 && terms[1].first > 0) std::swap(terms[0], terms[1]);
        std::string e = (terms[0].first > 0 ? "" : "-") + terms[0].second;
        for (size_t i = 1; i < terms.size(); ++i) e += (terms[i].first > 0 ? " + " : " - ") + terms[i].second;
        return e;
    };
    MomExpr m;
    m.x = sum("kx", nullptr, "");
    m.y = sum("ky", nullptr, "");
    m.z = sum("kz", "Q.kexth", "");
    m.xl = sum("kxl", nullptr, cast);
    m.yl = sum("kyl", nullptr, cast);
    m.zl = sum("kzl", "Q.kextl", cast);
    m.ks = coef(0) > 0 ? "1.0f" : coef(0) < 0 ? "-1.0f" : "0.0f";
    return m;
}

// the remainder sums of momentum_expr as exact double-float expressions
// (FdDF; one error-free addition per further term)
MomExpr momentum_df_expr(uint32_t mask, int N) {
    auto coef = [&](int j) { return (int)(((int32_t)(mask << (30 - 2 * j))) >> 30); };
    auto sum = [&](const char *comp, const char *ext) {
        std::vector<std::pair<int, std::string>> terms;
        if (ext && coef(0)) terms.push_back({coef(0), ext});
        for (int j = 1; j <= N; ++j)
            if (coef(j)) terms.push_back({coef(j), std::string("V.") + comp + "[" + std::to_string(j - 1) + "]"});
        if (terms.empty()) return std::string("FdDF{0.0f, 0.0f}");
        std::string e = std::string("FdDF{") + (terms[0].first > 0 ? "" : "-") + terms[0].second + ", 0.0f}";
        for (size_t i = 1; i < terms.size(); ++i)
            e = "fd_df_addf(" + e + ", " + (terms[i].first > 0 ? "" : "-") + terms[i].second + ")";
        return e;
    };
    MomExpr m;
    m.xl = sum("kxl", nullptr);
    m.yl = sum("kyl", nullptr);
    m.zl = sum("kzl", "Q.kextl");
    return m;
}

// time difference t_a - t_b of a G leaf's interaction lines as (dxh, dxl)
std::string time_diff_expr(uint32_t la, uint32_t lb, const std::string &vt) {
    const std::string a = std::to_string(la), b = std::to_string(lb);
    if (la == lb) return "    const " + vt + " dxh = 0.0f, dxl = 0.0f;\n";
    if (lb == 0) return "    const " + vt + " dxh = V.t[" + a + "], dxl = V.tl[" + a + "];\n";
    if (la == 0) return "    const " + vt + " dxh = -V.t[" + b + "], dxl = -V.tl[" + b + "];\n";
    return "    " + vt + " dxh, dxl;\n    fd_time_diff(V.t[" + a + "], V.tl[" + a + "], V.t[" + b + "], V.tl[" + b +
           "], dxh, dxl);\n";
}

// Code computing the Taylor family of leaf word w into `nm` (an array of its
// (M + 1)(1 + dk) values, or an FdLeafOut with leaf_calls); acc receives the
// access prefix of value j ("nm[" or "nm.v[").
std::string leaf_block(uint64_t w, const std::string &nm, uint32_t op, int N, const std::string &vt, int leaf_calls,
                       std::string &acc) {
    std::ostringstream o;
    const uint32_t mask = fa(w);
    const int no = leaf_outputs(w);
    const int M = (int)((w >> 40) & 7u), dk = (int)((w >> 43) & 1u);
    const bool precise = op == OP_GLEAF && ((w >> FD_LEAF_PRECISE_BIT) & 1u);
    const uint32_t la = (uint32_t)(w >> 34) & 7u, lb = (uint32_t)(w >> 37) & 7u;
    const MomExpr me = momentum_expr(mask, N);
    const std::string hi = "    const " + vt + " pxh = " + me.x + ", pyh = " + me.y + ", pzh = " + me.z + ";\n";
    acc = nm + "[";
    if (precise) {
        // double-float family (the single G line of the order-1 diagram), per
        // sample (packed: per lane); the remainder sums exact as double-floats
        o << "  " << vt << " " << nm << "[" << no << "];\n  {\n" << hi << time_diff_expr(la, lb, vt);
        const int lanes = vt == "float" ? 1 : 2;
        for (int q = 0; q < lanes; ++q) {
            const std::string L = vt == "float" ? "" : ".v." + std::string(q ? "y" : "x");
            const MomExpr ml = momentum_df_expr(mask, N);
            auto lane = [&](const std::string &e) {
                if (vt == "float") return e;
                // packed operands: take this lane of every V member
                std::string r = e, out;
                size_t pos = 0;
                while (true) {
                    const size_t a = r.find("]", pos);
                    if (a == std::string::npos) break;
                    out += r.substr(pos, a + 1 - pos) + L;
                    pos = a + 1;
                }
                return out + r.substr(pos);
            };
            o << "    g_family_df(" << "pxh" << L << ", pyh" << L << ", pzh" << L << ", " << lane(ml.xl) << ", "
              << lane(ml.yl) << ", " << lane(ml.zl) << ", " << me.ks << ", dxh" << L << ", dxl" << L
              << ", Q.beta, Q.betal, Q.muh, Q.mul, " << M << ", " << dk << ", [&](int j, float v) { ";
            if (vt == "float")
                o << nm << "[j] = v; });\n";
            else
                o << nm << "[j].v." << (q ? "y" : "x") << " = v; });\n";
        }
        o << "  }\n";
        return o.str();
    }
    const std::string lo = "    const " + vt + " pxl = " + me.xl + ", pyl = " + me.yl + ", pzl = " + me.zl + ";\n";
    if (leaf_calls) {
        acc = nm + ".v[";
        o << "  FdLeafOut<" << no << "> " << nm << ";\n  {\n" << hi << lo;
        if (op == OP_GLEAF) {
            o << time_diff_expr(la, lb, "float")
              << "    const float eps = fd_eps(pxh, pyh, pzh, pxl, pyl, pzl, Q.muh, Q.mul);\n"
              << "    " << nm << " = g_leaf_fn<" << M << ", " << dk << ">(eps, pzh + pzl, " << me.ks
              << ", dxh, dxl, Q.beta);\n  }\n";
        } else {
            o << "    const float qx = pxh + pxl, qy = pyh + pyl, qz = pzh + pzl;\n"
              << "    const float q2 = fmaf(qx, qx, fmaf(qy, qy, qz * qz));\n"
              << "    " << nm << " = v_leaf_fn<" << M << ", " << dk << ">(q2, qz, " << me.ks << ", Q.Lam);\n  }\n";
        }
        return o.str();
    }
    o << "  " << vt << " " << nm << "[" << no << "];\n  {\n" << hi << lo;
    if (op == OP_GLEAF) {
        o << time_diff_expr(la, lb, vt) << "    const " << vt
          << " eps = fd_eps(pxh, pyh, pzh, pxl, pyl, pzl, Q.muh, Q.mul);\n"
          << "    g_family<" << vt << ">(eps, pzh + pzl, " << me.ks << ", dxh, dxl, " << vt << "(Q.beta), " << M << ", "
          << dk << ", [&](int j, " << vt << " v) { " << nm << "[j] = v; });\n  }\n";
    } else {
        o << "    const " << vt << " qx = pxh + pxl, qy = pyh + pyl, qz = pzh + pzl;\n"
          << "    const " << vt << " q2 = fd_fma(qx, qx, fd_fma(qy, qy, qz * qz));\n"
          << "    v_family<" << vt << ">(q2, qz, " << me.ks << ", Q.Lam, " << M << ", " << dk << ", [&](int j, " << vt
          << " v) { " << nm << "[j] = v; });\n  }\n";
    }
    return o.str();
}

// Executed FP32 work of one leaf family (for ranking the leaf cache's
// candidates): momentum sums, eps, Fermi factor and exponentials, the series.
double leaf_cost(uint64_t w) {
    const uint32_t mask = fa(w);
    int terms = 0;
    for (int j = 0; j < 7; ++j) terms += ((mask >> (2 * j)) & 3u) != 0;
    const int M = (int)((w >> 40) & 7u), dk = (int)((w >> 43) & 1u), Mx = M + dk;
    double c = 6.0 * std::max(terms - 1, 0);
    if ((w & 63u) == OP_GLEAF) {
        c += 36.0 + 3.0 * 8.0;                       // eps, Fermi factor, exponentials (an SFU op ~ 8)
        for (int k = 0; k < Mx; ++k) c += (k + 1) + 4;
        if (Mx)
            for (int j = 0; j <= Mx; ++j) c += j + 1;
    } else {
        c += 12.0 + 8.0 + Mx;
    }
    return c;
}

// sync_every > 0: a block barrier after every sync_every arithmetic
// statements, so that the warps of a CTA walk the (long, straight-line) code
// together and share the instruction-cache lines they fetch.  Every thread of
// the block executes every statement, so the barriers are uniform.
// leaf_calls: leaves call the out-of-line family functions instead of inlining them.
// vt: value type of the generated code, "float" (one sample) or "FdF2" (two
// samples in packed two-lane arithmetic; no out-of-line leaves).
using LeafCache = std::map<uint32_t, int>;   // leaf instruction -> first float of its values in the cache

std::string emit_slice(const Slice &s, int q, const std::vector<TIns> &ins, const std::vector<uint64_t> &words,
                       int N, int n_slots, const char *qual, int sync_every, int leaf_calls,
                       const std::string &vt = "float", const LeafCache *cache = nullptr, int lc_stride = 0) {
    static const LeafCache empty;
    const auto cache_end = empty.end();
    std::ostringstream o;
    std::vector<std::string> cur(n_slots + 1);
    cur[0] = "0.0f";
    cur[1] = "1.0f";
    for (int j = 0; j < N; ++j) cur[2 + j] = "V.t[" + std::to_string(j) + "]";
    o << qual << " " << vt << " fd_s" << q << "(const FdSVT<" << vt << ", " << N << "> &V, const FdPar &Q"
      << (cache ? ", const float *L" : "") << ") {\n";
    int k = 0, since_sync = 0;
    for (const auto &kv : s.keep) {
        const TIns &t = ins[kv.first];
        const uint64_t w = words[t.w];
        if (sync_every > 0 && since_sync >= sync_every) {
            o << "  __syncthreads();\n";
            since_sync = 0;
        }
        since_sync += t.op == OP_BUNDLE ? (int)__builtin_popcount(kv.second) : (t.op == OP_CONST ? 0 : 8);
        if (t.op == OP_BUNDLE) {
            std::vector<std::pair<uint32_t, std::string>> upd;
            for (uint32_t m = 0; m < t.n; ++m) {
                if (!(kv.second >> m & 1u)) continue;
                const uint64_t mw = words[t.w + 1 + m];
                const uint32_t d = mw & 0xFFFFu, a = (mw >> 16) & 0xFFFFu, b = (mw >> 32) & 0xFFFFu,
                               c = (uint32_t)(mw >> 48);
                const std::string nm = "v" + std::to_string(k++);
                if (b == 1)
                    o << "  const " << vt << " " << nm << " = " << cur[a] << " + " << cur[c] << ";\n";
                else if (c == 0)
                    o << "  const " << vt << " " << nm << " = " << cur[a] << " * " << cur[b] << ";\n";
                else
                    o << "  const " << vt << " " << nm << " = fd_fma(" << cur[a] << ", " << cur[b] << ", " << cur[c]
                      << ");\n";
                upd.push_back({d, nm});
            }
            for (auto &u : upd) cur[u.first] = u.second;
        } else if (t.op == OP_GLEAF || t.op == OP_VLEAF) {
            const uint32_t d = fd_(w);
            const int no = leaf_outputs(w);
            const std::string nm = "l" + std::to_string(k++);
            const auto hit = cache ? cache->find(kv.first) : cache_end;
            if (cache && hit != cache->end()) {
                // computed once per sample by fd_leaves: read from the leaf cache
                o << "  const float " << nm << "[" << no << "] = {";
                for (int j = 0; j < no; ++j)
                    o << (j ? ", " : "") << "L[" << (hit->second + j) * lc_stride << "]";
                o << "};\n";
                for (int j = 0; j < no; ++j) cur[d + j] = nm + "[" + std::to_string(j) + "]";
                continue;
            }
            std::string acc;
            o << leaf_block(w, nm, t.op, N, vt, leaf_calls, acc);
            for (int j = 0; j < no; ++j) cur[d + j] = acc + std::to_string(j) + "]";
        } else if (t.op == OP_CONST) {
            uint32_t bits = (uint32_t)(w >> 32);
            float f;
            memcpy(&f, &bits, 4);
            cur[fd_(w)] = fnum(f);
        }
    }
    o << "  return " << cur[fa(words[ins[s.racc].w])] << ";\n}\n";
    return o.str();
}

struct Program {
    std::vector<std::string> modules;   // module 0 holds the kernel
    int n_modules = 1;
    int lc_floats = 0;                  // leaf-cache floats per sample (shared memory: x threads x spt)
};

// A compilation unit: one slice, or every slice of one root (the slices are
// then inlined into one function, so the compiler shares their leaves).
struct Unit {
    std::vector<int> slices;
    int root = -1;
    double cost = 0;
};

Program emit_program_loop(const fd_graph &g, int T, int min_blocks, int max_modules, int spt, double unit_cap,
                          int leaf_calls, int pair, int sync_units, int sv_smem, int cross_roots, int leaf_cache,
                          int lc_global);

Program emit_program(const fd_graph &g, int T, int min_blocks, int max_modules, int root_units, int sync_every,
                     int leaf_calls, int spt = 1, int unit_cap = 6000, int pair = 0, int sv_smem = 0,
                     int cross_roots = 0, int leaf_cache = 0, int lc_global = 0) {
    if (spt > 1 || leaf_cache > 0)
        return emit_program_loop(g, T, min_blocks, max_modules, spt, (double)unit_cap, leaf_calls, pair, sync_every,
                                 sv_smem, cross_roots, leaf_cache, lc_global);
    const TapeHeader &h = g.hdr;
    const int N = (int)h.order, DIM = (int)h.dim, R = (int)h.n_roots;
    const std::vector<TIns> ins = decode(g.h_tape);
    std::vector<Slice> sl = make_slices(ins, g.h_tape, (int)h.n_slots);
    double total = 0;
    for (auto &s : sl) total += s.cost();
    std::vector<Unit> units;
    if (root_units) {
        for (size_t i = 0; i < sl.size(); ++i) {
            if (units.empty() || units.back().root != sl[i].root) {
                units.emplace_back();
                units.back().root = sl[i].root;
            }
            units.back().slices.push_back((int)i);
        }
        for (Unit &u : units) {
            std::vector<uint32_t> leaves;
            for (int i : u.slices) {
                u.cost += sl[i].n_fma;
                for (auto &kv : sl[i].keep)
                    if (ins[kv.first].op == OP_GLEAF || ins[kv.first].op == OP_VLEAF) leaves.push_back(kv.first);
            }
            std::sort(leaves.begin(), leaves.end());
            u.cost += 30.0 * (double)(std::unique(leaves.begin(), leaves.end()) - leaves.begin());
        }
    } else {
        for (size_t i = 0; i < sl.size(); ++i) {
            units.emplace_back();
            units.back().slices.push_back((int)i);
            units.back().cost = sl[i].cost();
        }
    }
    int n_mod = 1;
    if (total > kSingleModuleCost && max_modules > 1)
        n_mod = std::max(2, std::min(max_modules, (int)(total / 2500.0) + 1));
    // largest units first onto the least loaded module (module 0 also holds the kernel)
    std::vector<int> mod_of(units.size(), 0);
    if (n_mod > 1) {
        std::vector<int> order(units.size());
        for (size_t i = 0; i < units.size(); ++i) order[i] = (int)i;
        std::sort(order.begin(), order.end(), [&](int a, int b) { return units[a].cost > units[b].cost; });
        std::vector<double> load(n_mod, 0.0);
        load[0] = 300.0;
        for (int i : order) {
            const int m = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            mod_of[i] = m;
            load[m] += units[i].cost;
        }
        // drop empty modules (fewer units than modules), keeping the kernel module 0
        std::vector<int> remap(n_mod, -1), used(n_mod, 0);
        used[0] = 1;
        for (int m : mod_of) used[m] = 1;
        int k = 0;
        for (int m = 0; m < n_mod; ++m)
            if (used[m]) remap[m] = k++;
        for (int &m : mod_of) m = remap[m];
        n_mod = k;
    }
    const bool multi = n_mod > 1;
    const bool by_root = multi && root_units;
    Program P;
    P.n_modules = n_mod;
    P.modules.assign(n_mod, std::string());
    std::vector<std::ostringstream> src(n_mod);
    for (int m = 0; m < n_mod; ++m)
        src[m] << "// generated from a validated fdcore tape: order " << N << ", " << R << " roots, " << sl.size()
               << " root-accumulate slices\n#include \"fd_jit_rt.cuh\"\nusing FdSV = FdSVT<float, " << N << ">;\n";
    const char *slice_qual = (multi && !by_root) ? "extern \"C\" __device__ __noinline__" : "static __device__ __forceinline__";
    for (size_t u = 0; u < units.size(); ++u) {
        const int m = mod_of[u];
        for (int i : units[u].slices) {
            if (multi && !by_root && m != 0)
                src[0] << "extern \"C\" __device__ float fd_s" << i << "(const FdSV &V, const FdPar &Q);\n";
            src[m] << emit_slice(sl[i], i, ins, g.h_tape, N, (int)h.n_slots, slice_qual, sync_every, leaf_calls);
        }
        if (by_root) {
            const int r = units[u].root;
            if (m != 0)
                src[0] << "extern \"C\" __device__ float2 fd_r" << r
                       << "(const FdSV &V, const FdPar &Q, const float *cs, const float *sn);\n";
            src[m] << "extern \"C\" __device__ __noinline__ float2 fd_r" << r
                   << "(const FdSV &V, const FdPar &Q, const float *cs, const float *sn) {\n  float re = 0.0f, im = 0.0f, v;\n";
            for (int i : units[u].slices)
                src[m] << "  v = fd_s" << i << "(V, Q); re = fmaf(v, cs[" << sl[i].line << "], re); im = fmaf(v, sn["
                       << sl[i].line << "], im);\n";
            src[m] << "  return make_float2(re, im);\n}\n";
        }
    }
    // body: roots in flush order, each the sum of its slices times exp(i pi x_line)
    std::ostringstream b;
    b << "struct FdBody {\n  template <class K>\n  static __device__ __forceinline__ void run(const FdSV &V, const FdPar &Q, const float (&cs)["
      << N << "], const float (&sn)[" << N << "], K &k) {\n";
    size_t si = 0;
    for (const TIns &t : ins) {
        if (t.op != OP_RFLUSH) continue;
        const int r = (int)fd_(g.h_tape[t.w]);
        const uint32_t rt = g.h_roots[2 * r];
        const std::string fl = "k.template flush<" + std::to_string(r) + ", " + std::to_string(rt & 255u) + ", " +
                               (((rt >> 24) & 255u) ? "1" : "0") + ">";
        const bool has = si < sl.size() && sl[si].root == r;
        if (by_root && has) {
            b << "    {\n      const float2 z = fd_r" << r << "(V, Q, cs, sn);\n      " << fl << "(z.x, z.y);\n    }\n";
            while (si < sl.size() && sl[si].root == r) ++si;
            continue;
        }
        b << "    {\n      float re = 0.0f, im = 0.0f, v;\n";
        for (; si < sl.size() && sl[si].root == r; ++si)
            b << "      v = fd_s" << si << "(V, Q); re = fmaf(v, cs[" << sl[si].line << "], re); im = fmaf(v, sn["
              << sl[si].line << "], im);\n";
        b << "      " << fl << "(re, im);\n    }\n";
    }
    b << "  }\n};\n";
    src[0] << b.str();
    src[0] << "extern \"C\" __global__ void __launch_bounds__(" << T << ", " << min_blocks
           << ") fd_jit_kernel(const __grid_constant__ EvalArgs A) {\n  jit_main<FdBody, " << N << ", " << DIM << ", "
           << R << ", " << T << ">(A);\n}\n";
    for (int m = 0; m < n_mod; ++m) P.modules[m] = src[m].str();
    return P;
}

// Emission with P > 1 samples per thread: compilation units (a root, or one
// slice of a root whose cost exceeds unit_cap) loop over the P samples.
// sync_units != 0: a block barrier after every unit call, so that the warps of
// a CTA run the same unit together and share its instruction-cache lines
// (every thread calls every unit: the barriers are uniform).
// sv_smem != 0: the per-sample inputs in shared memory, sample p of a thread
// at V[p * T] (otherwise a local array, V[p]).
// cross_roots != 0: units pack consecutive slices across root boundaries (the
// leaves that neighbouring roots share are computed once per unit); each
// unit adds into the accumulators of the roots it touches, and every root is
// flushed after all units.
Program emit_program_loop(const fd_graph &g, int T, int min_blocks, int max_modules, int spt, double unit_cap,
                          int leaf_calls, int pair, int sync_units, int sv_smem, int cross_roots, int leaf_cache,
                          int lc_global) {
    const std::string vs = sv_smem ? " * " + std::to_string(T) : "";
    const TapeHeader &h = g.hdr;
    const int N = (int)h.order, DIM = (int)h.dim, R = (int)h.n_roots;
    const std::vector<TIns> ins = decode(g.h_tape);
    std::vector<Slice> sl = make_slices(ins, g.h_tape, (int)h.n_slots);
    double total = 0;
    for (auto &s : sl) total += s.cost();
    // units: consecutive slices of one root packed while the unit's cost
    // (FMAs + 30 per distinct leaf, the leaves shared inside the unit) stays
    // within unit_cap; a unit's code is re-executed for the spt samples
    std::vector<Unit> units;
    auto unit_cost = [&](const std::vector<int> &slices) {
        std::vector<uint32_t> leaves;
        double c = 0;
        for (int i : slices) {
            c += sl[i].n_fma;
            for (auto &kv : sl[i].keep)
                if (ins[kv.first].op == OP_GLEAF || ins[kv.first].op == OP_VLEAF) leaves.push_back(kv.first);
        }
        std::sort(leaves.begin(), leaves.end());
        return c + 30.0 * (double)(std::unique(leaves.begin(), leaves.end()) - leaves.begin());
    };
    for (size_t i = 0; i < sl.size(); ++i) {
        if (!units.empty() && (cross_roots || units.back().root == sl[i].root)) {
            std::vector<int> grown = units.back().slices;
            grown.push_back((int)i);
            const double c = unit_cost(grown);
            if (c <= unit_cap) {
                units.back().slices = grown;
                units.back().cost = c;
                continue;
            }
        }
        units.emplace_back();
        units.back().root = sl[i].root;
        units.back().slices.push_back((int)i);
        units.back().cost = unit_cost(units.back().slices);
    }
    // leaf cache: families used by several units, computed once per sample
    // by fd_leaves into shared memory [float][sample][thread] (stride spt T)
    // and read by the units, the most work saved per float first, up to
    // leaf_cache floats per sample
    LeafCache cache;
    int lc_floats = 0;
    std::vector<uint32_t> cached;
    if (leaf_cache > 0) {
        std::map<uint32_t, int> uses;
        for (const Unit &u : units) {
            std::vector<uint32_t> ls;
            for (int i : u.slices)
                for (auto &kv : sl[i].keep)
                    if (ins[kv.first].op == OP_GLEAF || ins[kv.first].op == OP_VLEAF) ls.push_back(kv.first);
            std::sort(ls.begin(), ls.end());
            ls.erase(std::unique(ls.begin(), ls.end()), ls.end());
            for (uint32_t l : ls) ++uses[l];
        }
        std::vector<std::pair<double, uint32_t>> cand;
        for (auto &kv : uses) {
            if (kv.second < 2) continue;
            const uint64_t w = g.h_tape[ins[kv.first].w];
            cand.push_back({leaf_cost(w) * (kv.second - 1) / leaf_outputs(w), kv.first});
        }
        std::sort(cand.begin(), cand.end(), [](const std::pair<double, uint32_t> &a, const std::pair<double, uint32_t> &b) {
            return a.first > b.first || (a.first == b.first && a.second < b.second);
        });
        for (auto &c : cand) {
            const int wd = leaf_outputs(g.h_tape[ins[c.second].w]);
            if (lc_floats + wd > leaf_cache) continue;
            cached.push_back(c.second);
            lc_floats += wd;
        }
        std::sort(cached.begin(), cached.end());
        int off = 0;
        for (uint32_t c : cached) {
            cache[c] = off;
            off += leaf_outputs(g.h_tape[ins[c].w]);
        }
    }
    const LeafCache *cp = lc_floats ? &cache : nullptr;
    const int lc_stride = spt * T;
    int n_mod = 1;
    if (total > kSingleModuleCost && max_modules > 1)
        n_mod = std::max(2, std::min(max_modules, (int)(total / 2500.0) + 1));
    std::vector<int> mod_of(units.size(), 0);
    if (n_mod > 1) {
        std::vector<int> order(units.size());
        for (size_t i = 0; i < units.size(); ++i) order[i] = (int)i;
        std::sort(order.begin(), order.end(), [&](int a, int b) { return units[a].cost > units[b].cost; });
        std::vector<double> load(n_mod, 0.0);
        load[0] = 300.0;
        for (int i : order) {
            const int m = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            mod_of[i] = m;
            load[m] += units[i].cost;
        }
        std::vector<int> remap(n_mod, -1), used(n_mod, 0);
        used[0] = 1;
        for (int m : mod_of) used[m] = 1;
        int k = 0;
        for (int m = 0; m < n_mod; ++m)
            if (used[m]) remap[m] = k++;
        for (int &m : mod_of) m = remap[m];
        n_mod = k;
    }
    const bool multi = n_mod > 1;
    Program Pg;
    Pg.n_modules = n_mod;
    Pg.lc_floats = lc_floats;
    Pg.modules.assign(n_mod, std::string());
    std::vector<std::ostringstream> src(n_mod);
    for (int m = 0; m < n_mod; ++m)
        src[m] << "// generated from a validated fdcore tape: order " << N << ", " << R << " roots, " << sl.size()
               << " root-accumulate slices, " << spt << " samples per thread" << (pair ? " in packed pairs" : "")
               << "\n#include \"fd_jit_rt.cuh\"\nusing FdSV = FdSVT<float, " << N << ">;\n";
    const char *unit_qual = multi ? "extern \"C\" __device__ __noinline__" : "static __device__ __noinline__";
    const std::string sig =
        "(const FdSV *V, FdPar Q, const float *LC, const float *cs, const float *sn, float *re, float *im)";
    const std::string lcarg = cp ? ", LC + p * " + std::to_string(T) : "";
    // the leaf phase: every cached family of the thread's spt samples
    if (cp) {
        std::ostringstream lf;
        lf << "static __device__ __noinline__ void fd_leaves(const FdSV *Vb, FdPar Q, float *LC) {\n#pragma unroll 1\n"
              "  for (int p = 0; p < " << spt << "; ++p) {\n    const FdSV &V = Vb[p" << vs << "];\n    float *L = LC + p * "
           << T << ";\n";
        int k = 0;
        for (uint32_t c : cached) {
            const uint64_t w = g.h_tape[ins[c].w];
            const std::string nm = "c" + std::to_string(k++);
            std::string acc;
            lf << leaf_block(w, nm, ins[c].op, N, "float", 0, acc);
            const int off = cache.at(c);
            for (int j = 0; j < leaf_outputs(w); ++j)
                lf << "  L[" << (off + j) * lc_stride << "] = " << acc << j << "];\n";
        }
        lf << "  }\n}\n";
        src[0] << lf.str();
    }
    if (cross_roots) {
        // re/im: [root][sample] accumulators of the whole graph
        for (size_t u = 0; u < units.size(); ++u) {
            const int m = mod_of[u];
            for (int i : units[u].slices)
                src[m] << emit_slice(sl[i], i, ins, g.h_tape, N, (int)h.n_slots, "static __device__ __forceinline__",
                                     0, leaf_calls, pair ? "FdF2" : "float", cp, lc_stride);
            if (multi && m != 0) src[0] << "extern \"C\" __device__ void fd_u" << u << sig << ";\n";
            const std::vector<int> &us = units[u].slices;
            src[m] << unit_qual << " void fd_u" << u << sig << " {\n#pragma unroll 1\n  for (int p = 0; p < " << spt
                   << (pair ? "; p += 2) {\n    const auto W = fd_pack(V[p" + vs + "], V[(p + 1)" + vs + "]);\n"
                            : "; ++p) {\n")
                   << "    " << (pair ? "FdF2" : "float") << " v;\n";
            for (size_t a = 0; a < us.size();) {
                const int r = sl[us[a]].root;
                src[m] << "    {\n      " << (pair ? "FdF2" : "float") << " r = 0.0f, i = 0.0f;\n";
                for (; a < us.size() && sl[us[a]].root == r; ++a) {
                    const int i = us[a];
                    const std::string c0 = "p * " + std::to_string(N) + " + " + std::to_string(sl[i].line);
                    if (pair) {
                        const std::string c1 = "(p + 1) * " + std::to_string(N) + " + " + std::to_string(sl[i].line);
                        src[m] << "      v = fd_s" << i << "(W, Q); r = fd_fma(v, FdF2(cs[" << c0 << "], cs[" << c1
                               << "]), r); i = fd_fma(v, FdF2(sn[" << c0 << "], sn[" << c1 << "]), i);\n";
                    } else {
                        src[m] << "      v = fd_s" << i << "(V[p" << vs << "], Q" << lcarg << "); r = fmaf(v, cs[" << c0
                               << "], r); i = fmaf(v, sn[" << c0 << "], i);\n";
                    }
                }
                const std::string o = std::to_string(r * spt) + " + p";
                if (pair)
                    src[m] << "      re[" << o << "] += r.v.x;\n      re[" << o << " + 1] += r.v.y;\n      im[" << o
                           << "] += i.v.x;\n      im[" << o << " + 1] += i.v.y;\n    }\n";
                else
                    src[m] << "      re[" << o << "] += r;\n      im[" << o << "] += i;\n    }\n";
            }
            src[m] << "  }\n}\n";
        }
        std::ostringstream b;
        b << "struct FdBody {\n  template <class K>\n  static __device__ __forceinline__ void run(const FdSV *V, "
             "const FdPar &Q, float *LC, const float *cs, const float *sn, K *k) {\n"
          << (cp ? "    fd_leaves(V, Q, LC);\n" : "") << "    float re["
          << R * spt << "], im[" << R * spt << "];\n#pragma unroll\n    for (int q = 0; q < " << R * spt
          << "; ++q) re[q] = im[q] = 0.0f;\n";
        for (size_t u = 0; u < units.size(); ++u)
            b << "    fd_u" << u << "(V, Q, LC, cs, sn, re, im);\n" << (sync_units ? "    __syncthreads();\n" : "");
        for (const TIns &t : ins) {
            if (t.op != OP_RFLUSH) continue;
            const int r = (int)fd_(g.h_tape[t.w]);
            const uint32_t rt = g.h_roots[2 * r];
            b << "    flush_samples<" << r << ", " << (rt & 255u) << ", " << (((rt >> 24) & 255u) ? 1 : 0) << ", " << spt
              << ", " << N << ">(k, re + " << r * spt << ", im + " << r * spt << ");\n";
        }
        b << "  }\n};\n";
        src[0] << b.str();
        src[0] << "extern \"C\" __global__ void __launch_bounds__(" << T << ", " << min_blocks
               << ") fd_jit_kernel(const __grid_constant__ EvalArgs A) {\n  jit_main_loop<FdBody, " << N << ", " << DIM
               << ", " << R << ", " << T << ", " << spt << ", " << (sv_smem ? T : 1) << ", " << lc_floats
               << ", " << (lc_global && lc_floats ? "true" : "false")
               << ">(A);\n}\n";
        for (int m = 0; m < n_mod; ++m) Pg.modules[m] = src[m].str();
        return Pg;
    }
    for (size_t u = 0; u < units.size(); ++u) {
        const int m = mod_of[u];
        for (int i : units[u].slices)
            src[m] << emit_slice(sl[i], i, ins, g.h_tape, N, (int)h.n_slots, "static __device__ __forceinline__", 0,
                                 leaf_calls, pair ? "FdF2" : "float", cp, lc_stride);
        if (multi && m != 0) src[0] << "extern \"C\" __device__ void fd_u" << u << sig << ";\n";
        if (pair) {
            // samples p and p + 1 in the two lanes of packed arithmetic
            src[m] << unit_qual << " void fd_u" << u << sig << " {\n#pragma unroll 1\n  for (int p = 0; p < " << spt
                   << "; p += 2) {\n    const auto W = fd_pack(V[p" << vs << "], V[(p + 1)" << vs
                   << "]);\n    FdF2 r = 0.0f, i = 0.0f, v;\n";
            for (int i : units[u].slices) {
                const std::string c0 = "p * " + std::to_string(N) + " + " + std::to_string(sl[i].line);
                const std::string c1 = "(p + 1) * " + std::to_string(N) + " + " + std::to_string(sl[i].line);
                src[m] << "    v = fd_s" << i << "(W, Q); r = fd_fma(v, FdF2(cs[" << c0 << "], cs[" << c1
                       << "]), r); i = fd_fma(v, FdF2(sn[" << c0 << "], sn[" << c1 << "]), i);\n";
            }
            src[m] << "    re[p] += r.v.x;\n    re[p + 1] += r.v.y;\n    im[p] += i.v.x;\n    im[p + 1] += i.v.y;\n"
                      "  }\n}\n";
            continue;
        }
        src[m] << unit_qual << " void fd_u" << u << sig << " {\n#pragma unroll 1\n  for (int p = 0; p < " << spt
               << "; ++p) {\n    float r = 0.0f, i = 0.0f, v;\n";
        for (int i : units[u].slices)
            src[m] << "    v = fd_s" << i << "(V[p" << vs << "], Q" << lcarg << "); r = fmaf(v, cs[p * " << N << " + "
                   << sl[i].line
                   << "], r); i = fmaf(v, sn[p * " << N << " + " << sl[i].line << "], i);\n";
        src[m] << "    re[p] += r;\n    im[p] += i;\n  }\n}\n";
    }
    std::ostringstream b;
    b << "struct FdBody {\n  template <class K>\n  static __device__ __forceinline__ void run(const FdSV *V, const FdPar &Q, "
         "float *LC, const float *cs, const float *sn, K *k) {\n"
      << (cp ? "    fd_leaves(V, Q, LC);\n" : "");
    for (const TIns &t : ins) {
        if (t.op != OP_RFLUSH) continue;
        const int r = (int)fd_(g.h_tape[t.w]);
        const uint32_t rt = g.h_roots[2 * r];
        b << "    {\n      float re[" << spt << "], im[" << spt << "];\n#pragma unroll\n      for (int p = 0; p < "
          << spt << "; ++p) re[p] = im[p] = 0.0f;\n";
        for (size_t u = 0; u < units.size(); ++u)
            if (units[u].root == r)
                b << "      fd_u" << u << "(V, Q, LC, cs, sn, re, im);\n" << (sync_units ? "      __syncthreads();\n" : "");
        b << "      flush_samples<" << r << ", " << (rt & 255u) << ", " << (((rt >> 24) & 255u) ? 1 : 0) << ", "
          << spt << ", " << N << ">(k, re, im);\n    }\n";
    }
    b << "  }\n};\n";
    src[0] << b.str();
    src[0] << "extern \"C\" __global__ void __launch_bounds__(" << T << ", " << min_blocks
           << ") fd_jit_kernel(const __grid_constant__ EvalArgs A) {\n  jit_main_loop<FdBody, " << N << ", " << DIM
           << ", " << R << ", " << T << ", " << spt << ", " << (sv_smem ? T : 1) << ", " << lc_floats
               << ", " << (lc_global && lc_floats ? "true" : "false")
           << ">(A);\n}\n";
    for (int m = 0; m < n_mod; ++m) Pg.modules[m] = src[m].str();
    return Pg;
}

uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ull) {
    const uint8_t *b = (const uint8_t *)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct CompileOut {
    std::vector<char> cubin;
    std::string log;
    bool ok = false;
};

void compile_module(const std::string &src, int m, bool rdc, int maxrreg, CompileOut &out) {
    const Rtc &R = rtc();
    void *prog = nullptr;
    const char *hdrs[1] = {kRuntimeHeader};
    const char *names[1] = {"fd_jit_rt.cuh"};
    const std::string nm = "fd_jit_mod" + std::to_string(m) + ".cu";
    if (R.create(&prog, src.c_str(), nm.c_str(), 1, hdrs, names) != 0) {
        out.log = "nvrtcCreateProgram failed";
        return;
    }
    const std::string rr = "--maxrregcount=" + std::to_string(maxrreg);
    std::vector<const char *> opts = {"-arch=sm_103a", "-std=c++17", rr.c_str()};
    if (rdc) opts.push_back("-rdc=true");
    const int st = R.compile(prog, (int)opts.size(), opts.data());
    size_t ls = 0;
    R.log_size(prog, &ls);
    if (ls > 1) {
        out.log.resize(ls);
        R.log(prog, &out.log[0]);
    }
    if (st == 0) {
        size_t cs = 0;
        R.cubin_size(prog, &cs);
        out.cubin.resize(cs);
        R.cubin(prog, out.cubin.data());
        out.ok = cs > 0;
    }
    R.destroy(&prog);
}

fd_status build_cubin(const Program &P, int maxrreg, std::vector<char> &cubin) {
    const Rtc &R = rtc();
    if (!R.ok) return fd::set_error(FD_ENOTSUP, "run-time compilation unavailable: " + R.why);
    const bool rdc = P.n_modules > 1;
    std::vector<CompileOut> outs(P.n_modules);
    std::vector<std::thread> th;
    for (int m = 0; m < P.n_modules; ++m)
        th.emplace_back(compile_module, std::cref(P.modules[m]), m, rdc, maxrreg, std::ref(outs[m]));
    for (auto &t : th) t.join();
    for (int m = 0; m < P.n_modules; ++m)
        if (!outs[m].ok)
            return fd::set_error(FD_ENOTSUP, "NVRTC failed on module " + std::to_string(m) + ": " +
                                                 outs[m].log.substr(0, 4000));
    if (!rdc) {
        cubin = std::move(outs[0].cubin);
        return FD_OK;
    }
    void *lk = nullptr;
    const char *lopts[1] = {"-arch=sm_103a"};
    if (R.l_create(&lk, 1, lopts) != 0) return fd::set_error(FD_ENOTSUP, "nvJitLinkCreate failed");
    int st = 0;
    for (int m = 0; m < P.n_modules && st == 0; ++m) {
        const std::string nm = "fd_jit_mod" + std::to_string(m);
        st = R.l_add(lk, 1 /* NVJITLINK_INPUT_CUBIN */, outs[m].cubin.data(), outs[m].cubin.size(), nm.c_str());
    }
    if (st == 0) st = R.l_complete(lk);
    if (st != 0) {
        size_t ls = 0;
        R.l_log_size(lk, &ls);
        std::string log(ls, '\0');
        if (ls) R.l_log(lk, &log[0]);
        R.l_destroy(&lk);
        return fd::set_error(FD_ENOTSUP, "nvJitLink failed: " + log.substr(0, 4000));
    }
    size_t cs = 0;
    R.l_cubin_size(lk, &cs);
    cubin.resize(cs);
    R.l_cubin(lk, cubin.data());
    R.l_destroy(&lk);
    return FD_OK;
}

}  // namespace

fd_status jit_launch(const fd_graph *g, EvalArgs &args, cudaStream_t stream) {
    int dev = 0, n_sm = 0;
    FD_CHECK_CUDA(cudaGetDevice(&dev));
    FD_CHECK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    // tile histograms in shared memory when every adapting instance's grid
    // fits and a tile holds at least 4 samples per bin (the end-of-tile flush
    // then costs at most a quarter of the per-sample global atomics it replaces)
    int hist_floats = 0, bins_max = 0;
    for (int j = 0; j < args.n_inst; ++j)
        if (args.inst[j].hist) {
            hist_floats = std::max(hist_floats, args.inst[j].dim * args.inst[j].n_bins);
            bins_max = std::max(bins_max, args.inst[j].n_bins);
        }
    args.hist_smem = (hist_floats <= g->jit_hist_cap && args.tile >= 4 * (int64_t)bins_max) ? hist_floats : 0;
    const int items = args.n_inst * args.tiles_per_inst;
    const int grid = std::min(items, n_sm * g->jit_per_sm);   // <= the CTAs the global leaf cache holds
    args.lc_global = g->jit_lc;
    void *params[1] = {(void *)&args};
    FD_CHECK_CUDA(cudaLaunchKernel((const void *)g->jit_kernel, dim3(grid), dim3(g->jit_threads), params,
                                   (size_t)g->jit_sv_bytes + (size_t)args.hist_smem * sizeof(float), stream));
    return FD_OK;
}

namespace {
fd_status check_options(const fd_jit_options *o) {
    FD_REQUIRE(o, "options are required");
    FD_REQUIRE(o->threads == 64 || o->threads == 128 || o->threads == 256, "threads must be 64, 128 or 256");
    FD_REQUIRE(o->min_blocks >= 1 && o->min_blocks <= 8, "min_blocks must be in 1..8");
    FD_REQUIRE(o->max_modules >= 1 && o->max_modules <= 64, "max_modules must be in 1..64");
    FD_REQUIRE(o->sync_every >= 0, "sync_every must be >= 0");
    FD_REQUIRE(o->spt >= 1 && o->spt <= 16, "samples per thread must be in 1..16");
    FD_REQUIRE(o->unit_cap >= 0, "unit_cap must be >= 0");
    FD_REQUIRE(o->pair == 0 || (o->spt >= 2 && o->spt % 2 == 0 && !o->leaf_calls),
               "packed pairs need an even number of samples per thread and inlined leaves");
    FD_REQUIRE(o->sv_smem == 0 || o->spt >= 2, "per-sample inputs in shared memory need spt >= 2");
    FD_REQUIRE(o->cross_roots == 0 || o->spt >= 2, "units across roots need spt >= 2");
    FD_REQUIRE(o->leaf_cache >= 0 && o->leaf_cache <= 4096, "leaf_cache must be in 0..4096 floats per sample");
    FD_REQUIRE(o->leaf_cache == 0 || (!o->pair && !o->leaf_calls), "the leaf cache needs scalar, inlined leaves");
    FD_REQUIRE(o->lc_global == 0 || o->leaf_cache > 0, "lc_global needs a leaf cache");
    return FD_OK;
}

Program emit(const fd_graph &g, const fd_jit_options &o) {
    return emit_program(g, o.threads, o.min_blocks, o.max_modules, o.root_units, o.sync_every, o.leaf_calls, o.spt,
                        o.unit_cap, o.pair, o.sv_smem, o.cross_roots, o.leaf_cache, o.lc_global);
}
}  // namespace

extern "C" fd_status fd_jit_emit(const void *tape, size_t tape_len, const fd_jit_options *opt, int32_t module,
                                 char *buf, int64_t cap, int64_t *len, int32_t *n_modules) {
    FD_REQUIRE(tape, "tape is required");
    const fd_status so = check_options(opt);
    if (so != FD_OK) return so;
    fd_graph g;
    const fd_status st = graph_from_tape(tape, tape_len, g);
    if (st != FD_OK) return st;
    const Program P = emit(g, *opt);
    if (n_modules) *n_modules = P.n_modules;
    FD_REQUIRE(module >= 0 && module < P.n_modules, "module out of range");
    const std::string &s = P.modules[module];
    if (len) *len = (int64_t)s.size();
    if (buf && cap > 0) {
        const int64_t n = std::min<int64_t>(cap - 1, (int64_t)s.size());
        memcpy(buf, s.data(), (size_t)n);
        buf[n] = '\0';
    }
    return FD_OK;
}

extern "C" fd_status fd_graph_jit(fd_graph *g, const fd_jit_options *opt, const char *cache_dir) {
    FD_REQUIRE(g, "null graph");
    const fd_status so = check_options(opt);
    if (so != FD_OK) return so;
    const int threads = opt->threads, min_blocks = opt->min_blocks;
    int dev = 0;
    FD_CHECK_CUDA(cudaGetDevice(&dev));
    FD_REQUIRE(dev == g->device, "graph belongs to another device");
    const auto t0 = std::chrono::steady_clock::now();
    const int maxrreg = std::min(255, (65536 / (threads * min_blocks)) & ~7);
    const Program P = emit(*g, *opt);
    // cache key: generator version, launch shape, register cap and every module's source
    uint64_t key = fnv1a(&kJitVersion, sizeof kJitVersion);
    key = fnv1a(kRuntimeHeader, sizeof kRuntimeHeader, key);
    key = fnv1a(opt, sizeof *opt, key);
    key = fnv1a(&maxrreg, sizeof maxrreg, key);
    for (const auto &m : P.modules) key = fnv1a(m.data(), m.size(), key);
    std::string path;
    std::vector<char> cubin;
    if (cache_dir && cache_dir[0]) {
        char hex[32];
        snprintf(hex, sizeof hex, "%016llx", (unsigned long long)key);
        path = std::string(cache_dir) + "/fdjit_" + hex + ".cubin";
        std::ifstream f(path, std::ios::binary);
        if (f) cubin.assign(std::istreambuf_iterator<char>(f), std::istreambuf_iterator<char>());
    }
    if (cubin.empty()) {
        const fd_status st = build_cubin(P, maxrreg, cubin);
        if (st != FD_OK) return st;
        if (!path.empty()) {
            // private to this process and thread: a concurrent writer of the same
            // entry renames its own complete file
            const std::string tmp = path + ".tmp" + std::to_string((long long)getpid()) + "." +
                                    std::to_string(std::hash<std::thread::id>{}(std::this_thread::get_id()));
            std::ofstream f(tmp, std::ios::binary);
            f.write(cubin.data(), (std::streamsize)cubin.size());
            f.close();
            if (f) std::rename(tmp.c_str(), path.c_str());
        }
    }
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    FD_CHECK_CUDA(cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
    cudaError_t e = cudaLibraryGetKernel(&kern, lib, "fd_jit_kernel");
    cudaFuncAttributes attr;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&attr, (const void *)kern);
    if (e != cudaSuccess) {
        cudaLibraryUnload(lib);
        return fd::cuda_error(e, "loading the specialised kernel");
    }
    // dynamic shared memory: the per-sample inputs (sv_smem: threads x spt rows
    // of FdSV), then the tile histogram in what the resident CTAs leave free,
    // at most 96 KB so that the rest of the unified L1 keeps the per-thread
    // local arrays of the sample-loop variants
    const long sv_b = (opt->sv_smem ? (long)threads * opt->spt * (long)sizeof(float) * fd_sv_words((int)g->hdr.order)
                                    : 0) +
                      (opt->lc_global ? 0L : (long)threads * opt->spt * (long)sizeof(float) * P.lc_floats);
    int sm_total = 0, optin = 0, reserved = 0, hist_cap = 0;
    const bool have_attrs =
        cudaDeviceGetAttribute(&sm_total, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess;
    if (sv_b > 0) {
        cudaError_t es = have_attrs ? cudaSuccess : cudaErrorInvalidValue;
        if (es == cudaSuccess && sv_b + (long)attr.sharedSizeBytes > optin) es = cudaErrorInvalidValue;
        if (es == cudaSuccess)
            es = cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sv_b);
        if (es != cudaSuccess) {
            (void)cudaGetLastError();
            cudaLibraryUnload(lib);
            return fd::set_error(FD_EINVAL, "the per-sample inputs (" + std::to_string(sv_b) +
                                                " bytes per block) do not fit in shared memory");
        }
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)kern, threads, (size_t)sv_b) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        per_sm = std::max(1, 65536 / (std::max(attr.numRegs, 1) * threads));
    }
    per_sm = std::max(per_sm, 1);
    if (have_attrs) {
        const long free_b =
            std::min<long>((long)sm_total / per_sm - reserved, optin) - (long)attr.sharedSizeBytes - sv_b;
        const long cap_b = std::min<long>(free_b, 96 * 1024) & ~15L;
        if (cap_b > 0) {
            if (cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sv_b + cap_b)) == cudaSuccess)
                hist_cap = (int)(cap_b / (long)sizeof(float));
            else
                (void)cudaGetLastError();   // no tile histograms: global atomics only
        }
    }
    // global leaf cache: one region of threads x spt x floats per CTA the launch can place
    float *lcg = nullptr;
    int64_t lcg_floats = 0;
    if (opt->lc_global && P.lc_floats > 0) {
        int n_sm = 0;
        (void)cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        lcg_floats = (int64_t)n_sm * per_sm * threads * opt->spt * P.lc_floats;
        const cudaError_t ea = cudaMalloc(&lcg, (size_t)lcg_floats * sizeof(float));
        if (ea != cudaSuccess) {
            cudaLibraryUnload(lib);
            return fd::cuda_error(ea, "allocating the global leaf cache");
        }
    }
    if (g->jit_lib) cudaLibraryUnload(g->jit_lib);
    if (g->jit_lc) cudaFree(g->jit_lc);
    g->jit_lc = lcg;
    g->jit_lc_floats = lcg_floats;
    g->jit_per_sm = per_sm;
    g->jit_hist_cap = hist_cap;
    g->jit_sv_bytes = (int)sv_b;
    g->jit_lib = lib;
    g->jit_kernel = kern;
    g->jit_threads = threads;
    g->jit_min_blocks = min_blocks;
    g->jit_regs = attr.numRegs;
    g->jit_local_bytes = (int)attr.localSizeBytes;
    g->jit_modules = P.n_modules;
    g->jit_spt = opt->spt;
    g->jit_compile_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    g->jit_enabled = true;
    return FD_OK;
}

extern "C" fd_status fd_graph_jit_enable(fd_graph *g, int32_t on) {
    FD_REQUIRE(g, "null graph");
    FD_REQUIRE(!on || g->jit_kernel, "graph has no specialised kernel (call fd_graph_jit first)");
    g->jit_enabled = on != 0;
    return FD_OK;
}

extern "C" fd_status fd_graph_jit_info(const fd_graph *g, int32_t *info, double *compile_s) {
    FD_REQUIRE(g && info, "graph and info are required");
    info[0] = g->jit_threads;
    info[1] = g->jit_min_blocks;
    info[2] = g->jit_regs;
    info[3] = g->jit_local_bytes;
    info[4] = g->jit_modules;
    info[5] = g->jit_enabled ? 1 : 0;
    if (compile_s) *compile_s = g->jit_compile_s;
    return FD_OK;
}
