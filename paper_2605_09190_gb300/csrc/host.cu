// host.cu -- the C ABI of libaqmp.so: dictionary tables, device workspace,
// the level-synchronous quadtree loop (Algorithms 1-2) and the decoder entry
// (Algorithm 3).  All compute runs in this library's kernels; there is no
// CPU path.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/aqmp.h"
#include "common.cuh"
#include "kernels.h"
#include "selftest.h"
#include "haar_rows.cuh"
#include "code.h"

using namespace aqmp;

static_assert(sizeof(LeafRec) == sizeof(aqmp_leaf), "leaf record layout");
static_assert(sizeof(AtomRec) == sizeof(aqmp_atom), "atom record layout");

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? AQMP_E_OOM : AQMP_E_CUDA,         \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

// ---------------------------------------------------------------- FP64 bases
//
// The library's own generator (independent of the test oracle).
// DCT-II, Section 2.1 Eq. (1)-(2): C[k][m] = a_k cos(pi (2m + 1) k / (2N)),
// a_0 = sqrt(1/N), a_k = sqrt(2/N); the integer (2m + 1) k is formed first.
// Haar (Section 2.3 names it; standard orthonormal form): row 0 constant
// sqrt(1/N); row r >= 1 at scale s = 2^floor(log2 r), shift t = r - s has
// support [t N/s, (t+1) N/s), value +sqrt(s/N) on its first half and
// -sqrt(s/N) on its second.  Row 0 of both is the same expression, so the
// DCT DC atom and the Haar scaling atom are identical bit for bit.
void make_bases(int b, std::vector<double> &basis) {
    basis.assign(2 * (size_t)b * b, 0.0);
    double *C = basis.data(), *H = basis.data() + (size_t)b * b;
    // DCT-II row k is even (k even) or odd (k odd) about the block centre:
    // the second half mirrors the first exactly, so that the fixed-point rows
    // keep the symmetry the exact separable correlation relies on
    for (int k = 0; k < b; ++k) {
        const double ak = k == 0 ? std::sqrt(1.0 / b) : std::sqrt(2.0 / b);
        for (int m = 0; m < b / 2; ++m) {
            const long long num = (long long)(2 * m + 1) * k;
            const double v = k == 0 ? ak : ak * std::cos(M_PI * (double)num / (2.0 * b));
            C[k * b + m] = v;
            C[k * b + b - 1 - m] = (k & 1) ? -v : v;
        }
    }
    for (int m = 0; m < b; ++m) H[m] = std::sqrt(1.0 / b);
    for (int r = 1; r < b; ++r) {
        int scale = 1;                                   // 2^floor(log2 r)
        while (scale * 2 <= r) scale *= 2;
        const int t = r - scale;
        const int len = b / scale;
        const double v = std::sqrt((double)scale / b);
        for (int m = t * len; m < t * len + len / 2; ++m) H[r * b + m] = v;
        for (int m = t * len + len / 2; m < (t + 1) * len; ++m) H[r * b + m] = -v;
    }
}

// The exact SIMT correlation relies on these facts of the rows: DCT-II row
// k equals (-1)^k times its mirror image; Haar row r is v_r > 0 on the
// first of the halves haar_halves gives and -v_r on the second (row 0: v_0
// on both), zero elsewhere, with v_r the same for every row of one scale
// (the rows 2^j .. 2^(j+1) - 1).  Checked once per dictionary.
bool sep_rows_structured(int b, const std::vector<double> &basis) {
    const double *C = basis.data(), *H = basis.data() + (size_t)b * b;
    for (int k = 0; k < b; ++k) {
        for (int m = 0; m < b; ++m)
            if (C[k * b + b - 1 - m] != ((k & 1) ? -C[k * b + m] : C[k * b + m])) return false;
        int s, h;
        haar_halves(k, b, s, h);
        int first = k;                                   // first row of k's scale
        if (k > 0)
            while (first & (first - 1)) first &= first - 1;
        const double v = H[k * b + s];
        if (!(v > 0.0) || v != H[first * b]) return false;
        for (int m = 0; m < b; ++m) {
            const double want = m < s || m >= s + 2 * h ? 0.0 : (m < s + h || k == 0) ? v : -v;
            if (H[k * b + m] != want) return false;
        }
    }
    return true;
}

// Compensated dot product (Ogita-Rump-Oishi Dot2): result as accurate as if
// computed in twice the working precision, then rounded.
double dot2(const double *x, const double *y, int n) {
    double s = 0.0, c = 0.0;
    for (int i = 0; i < n; ++i) {
        const double p = x[i] * y[i];
        const double pe = std::fma(x[i], y[i], -p);
        const double t = s + p;
        const double z = t - s;
        const double se = (s - (t - z)) + (p - z);
        s = t;
        c += se + pe;
    }
    return s + c;
}

// ----------------------------------------------------------- tensor maps

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2-D BF16 tensor [rows][cols] (cols contiguous) read in boxes of
// box_rows x 64 elements with the 128-byte swizzle.
int encode_bf16_map(CUtensorMap *map, const void *base, unsigned long long rows, unsigned long long cols,
                    unsigned box_rows) {
    auto enc = tensor_map_encoder();
    if (!enc) return fail(AQMP_E_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * 2};
    cuuint32_t box[2] = {64, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(AQMP_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return AQMP_OK;
}

// 2-D byte tensor [rows][cols] (cols contiguous) read in boxes of box_rows x
// 128 bytes with the 128-byte swizzle (the FP8 operands).
int encode_u8_map(CUtensorMap *map, const void *base, unsigned long long rows, unsigned long long cols,
                  unsigned box_rows) {
    auto enc = tensor_map_encoder();
    if (!enc) return fail(AQMP_E_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols};
    cuuint32_t box[2] = {128, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(AQMP_E_CUDA, "cuTensorMapEncodeTiled (bytes) failed (%d)", (int)r);
    return AQMP_OK;
}

// ------------------------------------------------------------ context

// Bumped whenever a workspace buffer moves: captured graphs hold its
// addresses and are rebuilt after a move.
std::atomic<unsigned long long> g_ws_generation{0};

struct DeviceBuf {
    void *p = nullptr;
    size_t bytes = 0;
    ~DeviceBuf() { if (p) cudaFree(p); }
    int reserve(size_t want) {
        if (want <= bytes) return AQMP_OK;
        g_ws_generation.fetch_add(1);
        if (p) { cudaFree(p); p = nullptr; bytes = 0; }
        want = std::max<size_t>(want, 256);
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) { p = nullptr; return fail(AQMP_E_OOM, "cudaMalloc(%zu): %s", want, cudaGetErrorString(e)); }
        bytes = want;
        return AQMP_OK;
    }
};

// ------------------------------------------------------ kernel timing

struct Profiler {
    std::mutex mu;
    bool on = false;
    struct Pending { std::string name; cudaEvent_t a, b; bool owned = false; };
    std::vector<Pending> pending;
    // While this thread captures a graph its events are the graph's own
    // (created here, kept by the graph, queued again at every replay, never
    // pooled).
    static thread_local std::vector<Pending> *capture_to;
    std::string filter;                // time only kernels whose name starts with this
    std::vector<cudaEvent_t> pool;
    std::map<std::string, std::pair<unsigned long long, double>> totals;
    cudaEvent_t get() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    // Events around one launch; `launch` returns the launch's cudaError_t.
    template <class F>
    cudaError_t run(const std::string &name, cudaStream_t st, F &&launch) {
        if (!on || name.compare(0, filter.size(), filter) != 0) return launch();
        cudaEvent_t a = nullptr, b = nullptr;
        if (capture_to) {
            cudaEventCreate(&a);
            cudaEventCreate(&b);
        } else {
            a = get();
            b = get();
        }
        // in a graph, external event-record nodes: real records of the
        // events each time the node runs, so replays can be timed
        const unsigned flags = capture_to ? cudaEventRecordExternal : cudaEventRecordDefault;
        cudaEventRecordWithFlags(a, st, flags);
        cudaError_t e = launch();
        cudaEventRecordWithFlags(b, st, flags);
        if (capture_to) capture_to->push_back({name, a, b, true});
        else pending.push_back({name, a, b, false});
        return e;
    }
    // After the stream has been synchronised.
    void resolve() {
        for (auto &p : pending) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
                auto &t = totals[p.name];
                t.first += 1;
                t.second += ms;
            }
            if (!p.owned) {
                pool.push_back(p.a);
                pool.push_back(p.b);
            }
        }
        pending.clear();
    }
};
thread_local std::vector<Profiler::Pending> *Profiler::capture_to = nullptr;
Profiler g_prof;

std::string kname(const char *k, int b) { return std::string(k) + "_b" + std::to_string(b); }

// The exact separable correlation on the tensor-core path: the DCT-II family
// on the tensor cores, the Haar family on the SIMT pipes, where its rows' two
// constant halves reduce it to a summed-area computation with no contraction
// left to speed up.  Bit for bit the SIMT kernel's result for both families.
cudaError_t corr_sep_hybrid(const CorrArgs &ca, int b, cudaStream_t st) {
    const DictDev &d = *ca.d;
    const bool dct = d.nf == 2 || d.fam0 == 0, haar = d.nf == 2 || d.fam0 == 1;
    CorrArgs a = ca;
    cudaError_t e = cudaSuccess;
    if (dct) {
        a.fmask = 1;
        e = g_prof.run(kname("corr_septc_dct", b), st, [&] { return launch_corr_sep_tc(a, st); });
    }
    if (e == cudaSuccess && haar) {
        a.fmask = 2;
        e = g_prof.run(kname("corr_sep_haar", b), st, [&] { return launch_corr_sep_simt(a, st); });
    }
    return e;
}

// ------------------------------------------------------------ autotuner
//
// Choice points whose candidates give the same result bit for bit: the
// separable exact correlation on the tensor cores or on the integer SIMT
// path (K1, at the sides with a tensor-core kernel), and
// the pursuit's launch shape (K2: threads per leaf, or resident CTAs per SM
// at side 64).  Each is keyed by (kind, side,
// dictionary, precision, log2 capacity); its candidates are timed with CUDA
// events on the first calls (K1: both, twice each, within one encode, since
// recomputing the correlation is harmless; K2: alternately over encodes),
// and the one with the lowest timing is kept.  The lowest of two timings
// discards a kernel's first, cold launch.

struct Tuner {
    enum Kind { CORR = 0, MP = 1 };
    static constexpr int kSamples = 2;
    struct Slot {
        double best_ms[2] = {1e30, 1e30};
        int samples[2] = {0, 0};
        int chosen = -1;
    };
    struct Pending { Slot *slot; int cand; cudaEvent_t a, b; };
    std::map<std::array<int, 5>, Slot> slots;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    Slot &slot(int kind, int b, int dict, int prec, unsigned long long cap) {
        int lg = 0;
        while ((1ull << lg) < cap) ++lg;
        return slots[{kind, b, dict, prec, lg}];
    }
    static int next(const Slot &s) { return s.samples[1] < s.samples[0] ? 1 : 0; }
    cudaEvent_t get() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    template <class F>
    cudaError_t timed(Slot &s, int cand, cudaStream_t st, F &&launch) {
        cudaEvent_t a = get(), b = get();
        cudaEventRecord(a, st);
        cudaError_t e = launch();
        cudaEventRecord(b, st);
        pending.push_back({&s, cand, a, b});
        return e;
    }
    // After the stream has been synchronised.
    void resolve() {
        for (auto &p : pending) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
                Slot &s = *p.slot;
                s.best_ms[p.cand] = std::min(s.best_ms[p.cand], (double)ms);
                s.samples[p.cand] += 1;
                if (s.chosen < 0 && s.samples[0] >= kSamples && s.samples[1] >= kSamples)
                    s.chosen = s.best_ms[1] < s.best_ms[0] ? 1 : 0;
            }
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
    }
};

struct Dict {
    DictDev d{};
    DeviceBuf limbs, dh, dl, sh, sl, w, basis, basis64, sep, sepd, sepbf;
    CUtensorMap tmap_sd, tmap_sbf;
    CUtensorMap tmap;
    bool tables = false;         // fixed-point correlation tables built (16 M n B + 8 M n B)
    DeviceBuf dbf, sbf;          // reduced-precision form: bf16(D) and its row sums
    CUtensorMap tmap_bf;
    bool bf16 = false;
    DeviceBuf d8, s8;            // FP8 form: e4m3(D s_j), 1 / s_j and row sums
    CUtensorMap tmap_f8;
    bool fp8 = false;
};

struct Ctx {
    int device = -1;
    int num_sms = 0;
    int cc_major = 0, cc_minor = 0;
    std::mutex mu;
    std::map<int, std::unique_ptr<Dict>> dicts;
    DeviceBuf planes, staging, queues, Y, e0, c0, counters, ssim_ws, Y8, inv_sl, omp_L, mu_buf, ebound, fbq;
    DeviceBuf leaves_ws, atoms_ws, lo_ws, atom_leaf, cells, perm, new_off, order_status;   // emission -> canonical order
    bool gauss_ready = false;
    Tuner tuner;
    Counters *host_ctr = nullptr;             // pinned
    cudaMemPool_t out_pool = nullptr;         // encode outputs (aqmp_code arrays)
    unsigned char *host_call = nullptr;       // pinned: plane descriptors + output pointers
    size_t host_call_cap = 0;
    // Captured encodes, one per configuration (see aqmp_encode_planes).
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        unsigned long long generation = 0;
        std::vector<Profiler::Pending> prof;
    };
    std::map<std::vector<long long>, Graph> graphs;
    std::map<std::vector<long long>, int> seen;     // direct runs per configuration (-1: capture failed)
    cudaStream_t graph_stream = nullptr;            // graphs run here (capture needs a non-legacy stream)
    cudaEvent_t graph_in = nullptr, graph_out = nullptr;
    // device time of the last encode: events on the stream that runs its
    // kernels, recorded just before the first and just after the last
    cudaEvent_t dev_t0 = nullptr, dev_t1 = nullptr;
    float last_device_ms = -1.0f;
    void drop_graphs() {
        for (auto &kv : graphs) {
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            for (auto &p : kv.second.prof) {
                cudaEventDestroy(p.a);
                cudaEventDestroy(p.b);
            }
        }
        graphs.clear();
    }
};

std::mutex g_ctx_mu;
std::map<int, std::unique_ptr<Ctx>> g_ctx;

int get_ctx(Ctx **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(AQMP_E_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> g(g_ctx_mu);
    auto &slot = g_ctx[dev];
    if (!slot) {
        auto c = std::make_unique<Ctx>();
        c->device = dev;
        CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev));
        CK(cudaDeviceGetAttribute(&c->cc_major, cudaDevAttrComputeCapabilityMajor, dev));
        CK(cudaDeviceGetAttribute(&c->cc_minor, cudaDevAttrComputeCapabilityMinor, dev));
        if (c->cc_major != 10 || c->cc_minor != 3)
            return fail(AQMP_E_CUDA, "device %d is sm_%d%d; this library is built for sm_103a only", dev,
                        c->cc_major, c->cc_minor);
        CK(cudaMallocHost(&c->host_ctr, sizeof(Counters)));
        // the encode outputs come from a pool of the library's own, which
        // keeps freed blocks cached (the process-wide default pool, which
        // other code of the process may use, is left as it is)
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        CK(cudaMemPoolCreate(&c->out_pool, &props));
        unsigned long long keep = ~0ull;
        CK(cudaMemPoolSetAttribute(c->out_pool, cudaMemPoolAttrReleaseThreshold, &keep));
        slot = std::move(c);
    }
    *out = slot.get();
    return AQMP_OK;
}

int num_families(int dict_id) { return dict_id == AQMP_DICT_DCT_HAAR ? 2 : 1; }

// Tables of one (side, dictionary), built once per device: the FP32/FP64
// bases and W always; the fixed-point correlation tables (digit planes and
// (Dh, Dl): 24 M n bytes, 12.9 GB at side 128) only when `tables` is set,
// so that decoding and synthesis never build them; bf16(D) (2 M Kpad bytes)
// only when `bf16` is set (the reduced-precision form).
int get_dict(Ctx *c, int b, int dict_id, cudaStream_t st, Dict **out, bool tables = true, bool bf16 = false,
             bool fp8 = false) {
    const int key = b * 16 + dict_id;
    auto it = c->dicts.find(key);
    Dict *D = nullptr;
    if (it != c->dicts.end()) {
        D = it->second.get();
    } else {
        auto Dn = std::make_unique<Dict>();
        DictDev &d = Dn->d;
        d.b = b;
        d.n = b * b;
        d.nf = num_families(dict_id);
        d.M = d.nf * d.n;
        d.Mpad = std::max(128, (d.M + 127) / 128 * 128);
        d.Kpad = std::max(kKBlock, (d.n + kKBlock - 1) / kKBlock * kKBlock);
        int rc;
        if ((rc = Dn->w.reserve(sizeof(float) * 4 * (size_t)b * b))) return rc;
        if ((rc = Dn->basis.reserve(sizeof(float) * 2 * (size_t)b * b))) return rc;
        if ((rc = Dn->basis64.reserve(sizeof(double) * 2 * (size_t)b * b))) return rc;
        d.W = (float2 *)Dn->w.p;
        d.WT = d.W + b * b;
        d.basis = (float *)Dn->basis.p;
        d.fam0 = dict_id == AQMP_DICT_HAAR ? 1 : 0;

        std::vector<double> basis;
        make_bases(b, basis);
        if (!sep_rows_structured(b, basis)) return AQMP_E_UNSUPPORTED;

        // separable fixed-point dictionary: Bf = round(B 2^48) per 1-D row,
        // as 24-bit limbs (lo in [-2^23, 2^23), hi), its transpose, and the
        // row sums (both families; a few hundred KB at most)
        {
            const size_t bb = (size_t)b * b;
            std::vector<int32_t> limbs(2 * 2 * 2 * bb);            // Bs then BsT, (lo, hi) pairs
            std::vector<long long> rows(2 * (size_t)b, 0);
            for (int F = 0; F < 2; ++F)
                for (int p = 0; p < b; ++p)
                    for (int i = 0; i < b; ++i) {
                        const long long f = std::llrint(std::ldexp(basis[F * bb + (size_t)p * b + i], 48));
                        const long long lo = ((f + (1ll << 23)) & ((1ll << 24) - 1)) - (1ll << 23);
                        const long long hi = (f - lo) / (1ll << 24);
                        const size_t at = F * bb + (size_t)p * b + i, atT = 2 * bb + F * bb + (size_t)i * b + p;
                        limbs[2 * at] = (int32_t)lo;
                        limbs[2 * at + 1] = (int32_t)hi;
                        limbs[2 * atT] = (int32_t)lo;
                        limbs[2 * atT + 1] = (int32_t)hi;
                        rows[F * b + p] += f;
                    }
            int rc0;
            if ((rc0 = Dn->sep.reserve(sizeof(int32_t) * limbs.size() + sizeof(long long) * rows.size()))) return rc0;
            d.Bs = (int2 *)Dn->sep.p;
            d.BsT = d.Bs + 2 * bb;
            d.Rs = (long long *)(d.BsT + 2 * bb);
            CK(cudaMemcpyAsync(d.Bs, limbs.data(), sizeof(int32_t) * limbs.size(), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(d.Rs, rows.data(), sizeof(long long) * rows.size(), cudaMemcpyHostToDevice, st));
            if (corr_sep_tc_available(b, d.nf)) {
                // balanced base-2^8 digits d_s of Bf (s = 0..5) as BF16, in six
                // 128-row tiles (family F, digit pair u): row r of tile (F, u)
                // is row r mod b of digit 2u + r / b
                std::vector<__nv_bfloat16> dg(6 * 2 * bb);
                for (int F = 0; F < 2; ++F)
                    for (int r = 0; r < b; ++r)
                        for (int col = 0; col < b; ++col) {
                            long long f = std::llrint(std::ldexp(basis[F * bb + (size_t)r * b + col], 48));
                            for (int sd = 0; sd < 6; ++sd) {
                                long long dv = sd < 5 ? ((f + 128) & 255) - 128 : f;
                                f = (f - dv) >> 8;
                                const int u = sd >> 1, half = sd & 1;
                                dg[((size_t)(3 * F + u) * 2 * b + half * b + r) * b + col] = __float2bfloat16((float)dv);
                            }
                        }
                if ((rc0 = Dn->sepd.reserve(sizeof(__nv_bfloat16) * dg.size()))) return rc0;
                d.sepd = (__nv_bfloat16 *)Dn->sepd.p;
                CK(cudaMemcpyAsync(d.sepd, dg.data(), sizeof(__nv_bfloat16) * dg.size(), cudaMemcpyHostToDevice, st));
                if ((rc0 = encode_bf16_map(&Dn->tmap_sd, d.sepd, 6ull * 2 * b, b, 128))) return rc0;
                d.tmap_sepd = &Dn->tmap_sd;
                // the BF16 form with rescore (corr_sepbf_tc.cu): three
                // 128-row tiles of 1-D rows, [bf16(B_0); bf16(B_0 - bf16(B_0))],
                // the same for family 1, then [|B_0| ; |B_1|] rounded up to
                // BF16; and the row sums R[F][p] = sum_i B[F][p][i] as (hi, lo)
                std::vector<__nv_bfloat16> sb(3 * 2 * bb);
                std::vector<float2> rs(2 * (size_t)b);
                for (int F = 0; F < 2; ++F)
                    for (int r = 0; r < b; ++r) {
                        double sum = 0.0;
                        for (int col = 0; col < b; ++col) {
                            const double x = basis[F * bb + (size_t)r * b + col];
                            sum += x;
                            const __nv_bfloat16 hi = __float2bfloat16_rn((float)x);
                            const double rem = x - (double)__bfloat162float(hi);
                            const __nv_bfloat16 lo = __float2bfloat16_rn((float)rem);
                            float ax = (float)std::fabs(x);
                            if ((double)ax < std::fabs(x)) ax = std::nextafter(ax, INFINITY);
                            __nv_bfloat16 au = __float2bfloat16_rn(ax);
                            if (__bfloat162float(au) < ax) au = __float2bfloat16_ru(ax);
                            sb[((size_t)F * 2 * b + r) * b + col] = hi;
                            sb[((size_t)F * 2 * b + b + r) * b + col] = lo;
                            sb[((size_t)4 * b + F * b + r) * b + col] = au;
                        }
                        const float rh = (float)sum;
                        rs[(size_t)F * b + r] = make_float2(rh, (float)(sum - (double)rh));
                    }
                if ((rc0 = Dn->sepbf.reserve(sizeof(__nv_bfloat16) * sb.size() + sizeof(float2) * rs.size())))
                    return rc0;
                d.sepbf = (__nv_bfloat16 *)Dn->sepbf.p;
                d.Rbf = (float2 *)(d.sepbf + sb.size());
                CK(cudaMemcpyAsync(d.sepbf, sb.data(), sizeof(__nv_bfloat16) * sb.size(), cudaMemcpyHostToDevice, st));
                CK(cudaMemcpyAsync(d.Rbf, rs.data(), sizeof(float2) * rs.size(), cudaMemcpyHostToDevice, st));
                if ((rc0 = encode_bf16_map(&Dn->tmap_sbf, d.sepbf, 6ull * b, b, 128))) return rc0;
                d.tmap_sepbf = &Dn->tmap_sbf;
            }
        }
        // W = C H^T with exact structural zeros: entries below 2^-40 are the
        // rounding of an exact zero (e.g. W[p][0] = <C_p, H_0> = 0 for p > 0)
        std::vector<float> w(4 * (size_t)b * b);      // W then W^T, (hi, lo) interleaved
        const double *C = basis.data(), *H = basis.data() + (size_t)b * b;
        for (int p = 0; p < b; ++p)
            for (int q = 0; q < b; ++q) {
                double x = dot2(C + (size_t)p * b, H + (size_t)q * b, b);
                if (std::fabs(x) < 0x1p-40) x = 0.0;
                else if (std::fabs(x) < 1e-7)
                    return fail(AQMP_E_DICT, "cross-Gram entry W[%d][%d] = %g is neither zero nor well separated", p,
                                q, x);
                const float hi = (float)x, lo = (float)(x - (double)hi);
                w[2 * ((size_t)p * b + q)] = hi;                         // W[p][q]
                w[2 * ((size_t)p * b + q) + 1] = lo;
                w[2 * ((size_t)b * b + (size_t)q * b + p)] = hi;         // W^T[q][p]
                w[2 * ((size_t)b * b + (size_t)q * b + p) + 1] = lo;
            }
        CK(cudaMemcpyAsync(Dn->w.p, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(Dn->basis64.p, basis.data(), sizeof(double) * basis.size(), cudaMemcpyHostToDevice, st));
        CK(launch_basis_to_float((const double *)Dn->basis64.p, d.basis, 2 * b * b, st));
        if (dict_id == AQMP_DICT_HAAR) {
            // single Haar family: decoder table slot 0 must hold the Haar basis
            CK(cudaMemcpyAsync(d.basis, (const float *)Dn->basis.p + b * b, sizeof(float) * b * b,
                               cudaMemcpyDeviceToDevice, st));
        }
        CK(cudaStreamSynchronize(st));
        D = Dn.get();
        c->dicts[key] = std::move(Dn);
    }
    if (tables && !D->tables) {
        DictDev &d = D->d;
        int rc;
        if ((rc = D->limbs.reserve(sizeof(__nv_bfloat16) * (size_t)kLimbs * d.Mpad * d.Kpad))) return rc;
        if ((rc = D->dh.reserve(sizeof(int32_t) * (size_t)d.M * d.n))) return rc;
        if ((rc = D->dl.reserve(sizeof(int32_t) * (size_t)d.M * d.n))) return rc;
        if ((rc = D->sh.reserve(sizeof(long long) * d.M))) return rc;
        if ((rc = D->sl.reserve(sizeof(long long) * d.M))) return rc;
        d.limbs = (__nv_bfloat16 *)D->limbs.p;
        d.Dh = (int32_t *)D->dh.p;
        d.Dl = (int32_t *)D->dl.p;
        d.Sh = (long long *)D->sh.p;
        d.Sl = (long long *)D->sl.p;
        const int fam0 = dict_id == AQMP_DICT_HAAR ? 1 : 0;
        CK(build_fixed_tables_fam(d, (const double *)D->basis64.p, fam0, st));
        if ((rc = encode_bf16_map(&D->tmap, d.limbs, (unsigned long long)kLimbs * d.Mpad, d.Kpad, 128))) return rc;
        d.tmap_limbs = &D->tmap;
        CK(cudaStreamSynchronize(st));
        D->tables = true;
    }
    if (bf16 && !D->bf16) {
        DictDev &d = D->d;
        int rc;
        if ((rc = D->dbf.reserve(sizeof(__nv_bfloat16) * (size_t)d.Mpad * d.Kpad))) return rc;
        if ((rc = D->sbf.reserve(sizeof(float) * (size_t)d.M))) return rc;
        d.Dbf = (__nv_bfloat16 *)D->dbf.p;
        d.Sbf = (float *)D->sbf.p;
        const int fam0 = dict_id == AQMP_DICT_HAAR ? 1 : 0;
        CK(build_bf16_tables(d, (const double *)D->basis64.p, fam0, st));
        if ((rc = encode_bf16_map(&D->tmap_bf, d.Dbf, (unsigned long long)d.Mpad, d.Kpad, 128))) return rc;
        d.tmap_bf16 = &D->tmap_bf;
        CK(cudaStreamSynchronize(st));
        D->bf16 = true;
    }
    if (fp8 && !D->fp8) {
        DictDev &d = D->d;
        const int K8 = kpad_fp8(d.n);
        int rc;
        if ((rc = D->d8.reserve((size_t)d.Mpad * K8))) return rc;
        if ((rc = D->s8.reserve(sizeof(float) * 2 * (size_t)d.M))) return rc;
        d.D8 = (uint8_t *)D->d8.p;
        d.inv_s8 = (float *)D->s8.p;
        d.S8 = d.inv_s8 + d.M;
        CK(build_fp8_tables(d, (const double *)D->basis64.p, d.fam0, st));
        if ((rc = encode_u8_map(&D->tmap_f8, d.D8, (unsigned long long)d.Mpad, K8, 128))) return rc;
        d.tmap_fp8 = &D->tmap_f8;
        CK(cudaStreamSynchronize(st));
        D->fp8 = true;
    }
    *out = D;
    return AQMP_OK;
}

int check_params(const aqmp_params *p) {
    if (!p) return fail(AQMP_E_ARG, "params is NULL");
    if (!(p->rmse_tol >= 0.0f)) return fail(AQMP_E_ARG, "rmse_tol must be >= 0");
    if (p->cap_num < 0 || p->cap_den <= 0 || (long long)p->cap_num > (long long)p->cap_den)
        return fail(AQMP_E_ARG, "sparsity cap must satisfy 0 <= cap_num <= cap_den, cap_den > 0");
    if (!is_pow2(p->min_block) || !is_pow2(p->max_block) || p->min_block < 4 || p->max_block < p->min_block)
        return fail(AQMP_E_ARG, "block sizes must be powers of two with 4 <= min_block <= max_block");
    if (p->max_block > kMaxSide) return fail(AQMP_E_UNSUPPORTED, "max_block above %d is not built", kMaxSide);
    if (p->dict_id < 0 || p->dict_id > 2) return fail(AQMP_E_DICT, "unknown dictionary id %d", p->dict_id);
    if (p->precision != AQMP_PREC_EXACT && p->precision != AQMP_PREC_FP32 && p->precision != AQMP_PREC_BF16 &&
        p->precision != AQMP_PREC_FP8 && p->precision != AQMP_PREC_BF16_RESCORE)
        return fail(AQMP_E_UNSUPPORTED, "unknown precision %d", p->precision);
    return AQMP_OK;
}

}  // namespace

// Internal helpers shared with other translation units of the library.
namespace aqmp {
int set_error(int code, const char *msg) { return fail(code, "%s", msg); }
void fp64_bases(int b, std::vector<double> &basis) { make_bases(b, basis); }
int bf16_tensor_map(void *map, const void *base, unsigned long long rows, unsigned long long cols,
                    unsigned box_rows) {
    return encode_bf16_map(reinterpret_cast<CUtensorMap *>(map), base, rows, cols, box_rows);
}
int device_sm_count(int *sms) {
    Ctx *c;
    const int rc = get_ctx(&c);
    if (rc == AQMP_OK) *sms = c->num_sms;
    return rc;
}
}  // namespace aqmp

// ===================================================================== ABI


extern "C" {

const char *aqmp_last_error(void) { return g_last_error.c_str(); }

int aqmp_last_device_ms(double *ms) {
    g_last_error.clear();
    if (!ms) return fail(AQMP_E_ARG, "ms is NULL");
    Ctx *c;
    int rc;
    if ((rc = get_ctx(&c))) return rc;
    std::lock_guard<std::mutex> lock(c->mu);
    *ms = c->last_device_ms;
    return AQMP_OK;
}

int aqmp_autotune_read(aqmp_tune_entry *out, int max, int *n) {
    if (!n || (max > 0 && !out)) return fail(AQMP_E_ARG, "NULL argument");
    Ctx *c;
    int rc;
    if ((rc = get_ctx(&c))) return rc;
    std::lock_guard<std::mutex> lock(c->mu);
    int k = 0;
    for (const auto &kv : c->tuner.slots) {
        if (k < max) {
            aqmp_tune_entry &e = out[k];
            e.kind = kv.first[0];
            e.side = kv.first[1];
            e.dict_id = kv.first[2];
            e.precision = kv.first[3];
            e.capacity_log2 = kv.first[4];
            e.chosen = kv.second.chosen;
            for (int i = 0; i < 2; ++i) {
                e.samples[i] = kv.second.samples[i];
                e.best_ms[i] = kv.second.samples[i] ? kv.second.best_ms[i] : 0.0;
            }
        }
        ++k;
    }
    *n = k;
    return AQMP_OK;
}

void aqmp_autotune_reset(void) {
    Ctx *c;
    if (get_ctx(&c)) return;
    std::lock_guard<std::mutex> lock(c->mu);
    c->tuner.slots.clear();
    c->tuner.pending.clear();
    c->drop_graphs();                 // they embed the forgotten choices
    c->seen.clear();
}
const char *aqmp_version(void) { return "aqmp-gb300 0.1 (sm_103a)"; }

void aqmp_params_default(aqmp_params *p) {
    if (!p) return;
    p->rmse_tol = 2.0f;
    p->cap_num = 1;
    p->cap_den = 4;
    p->min_block = 4;
    p->max_block = 64;
    p->dict_id = AQMP_DICT_DCT_HAAR;
    p->precision = AQMP_PREC_EXACT;
    p->flags = 0;
}

int aqmp_num_atoms(int b, int dict_id) {
    if (!is_pow2(b) || dict_id < 0 || dict_id > 2) return AQMP_E_ARG;
    return num_families(dict_id) * b * b;
}

int aqmp_encode_planes(const aqmp_params *params, const aqmp_plane *planes, int n_planes, void *stream,
                       aqmp_code **out) {
    g_last_error.clear();
    if (!out) return fail(AQMP_E_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_params(params);
    if (rc) return rc;
    if (!planes || n_planes <= 0) return fail(AQMP_E_ARG, "no planes");
    const aqmp_params P = *params;
    const bool dev_in = (P.flags & AQMP_FLAG_INPUT_DEVICE) != 0;
    const bool simt = (P.flags & AQMP_FLAG_SIMT_GEMM) != 0;
    const bool tune = (P.flags & AQMP_FLAG_NO_AUTOTUNE) == 0;
    const bool alt_threads = (P.flags & AQMP_FLAG_ALT_THREADS) != 0;
    const bool omp = (P.flags & AQMP_FLAG_OMP) != 0;
    const bool bf16 = P.precision == AQMP_PREC_BF16;
    const bool fp8 = P.precision == AQMP_PREC_FP8;
    // the BF16 form with rescore: its own correlation and pursuit at the sides
    // a kernel for it serves (64), the exact form elsewhere
    const bool resc = P.precision == AQMP_PREC_BF16_RESCORE;
    if (omp) {
        if (P.max_block > 64 || P.precision != AQMP_PREC_EXACT)
            return fail(AQMP_E_UNSUPPORTED, "OMP needs max_block <= 64 and the exact precision");
        for (int b = P.max_block; b >= P.min_block; b >>= 1) {
            const long long kb = std::max<long long>(1, (long long)b * b * P.cap_num / P.cap_den);
            if (kb > omp_max_budget(b))
                return fail(AQMP_E_UNSUPPORTED, "OMP budget above %d atoms per leaf at side %d", omp_max_budget(b), b);
        }
    }
    unsigned long long npix = 0, roots = 0, staged = 0;
    for (int i = 0; i < n_planes; ++i) {
        const aqmp_plane &pl = planes[i];
        if (!pl.pixels || pl.height <= 0 || pl.width <= 0 || pl.pitch < pl.width)
            return fail(AQMP_E_ARG, "plane %d: bad pointer or shape", i);
        if (pl.height % P.max_block || pl.width % P.max_block)
            return fail(AQMP_E_SHAPE, "plane %d: %dx%d is not a multiple of max_block %d", i, pl.height,
                        pl.width, P.max_block);
        const float tol = pl.rmse_tol < 0.0f ? P.rmse_tol : pl.rmse_tol;
        if (!(tol >= 0.0f)) return fail(AQMP_E_ARG, "plane %d: bad tolerance", i);
        npix += (unsigned long long)pl.height * pl.width;
        roots += (unsigned long long)(pl.height / P.max_block) * (pl.width / P.max_block);
        staged += (unsigned long long)pl.height * pl.width;
    }
    if (npix / ((unsigned long long)P.min_block * P.min_block) > 0xffffffffull / 8)
        return fail(AQMP_E_UNSUPPORTED, "batch too large for 32-bit queues");

    Ctx *c;
    if ((rc = get_ctx(&c))) return rc;
    std::lock_guard<std::mutex> lock(c->mu);
    cudaStream_t st = (cudaStream_t)stream;

    const int nlev = ilog2(P.max_block) - ilog2(P.min_block) + 1;
    std::vector<Dict *> dicts(nlev);
    for (int l = 0; l < nlev; ++l)
        if ((rc = get_dict(c, P.max_block >> l, P.dict_id, st, &dicts[l], false, bf16, fp8))) return rc;

    // capacities
    std::vector<unsigned long long> cap(nlev), qoff(nlev + 1, 0);
    unsigned long long ymax = 0, cmax = 0, emax = 0, y8max = 0;
    for (int l = 0; l < nlev; ++l) {
        const int b = P.max_block >> l;
        cap[l] = npix / ((unsigned long long)b * b);
        qoff[l + 1] = qoff[l] + cap[l];
        ymax = std::max(ymax, cap[l] * dicts[l]->d.Kpad);
        y8max = std::max(y8max, cap[l] * (unsigned long long)kpad_fp8(dicts[l]->d.n));
        cmax = std::max(cmax, cap[l] * dicts[l]->d.M);
        emax = std::max(emax, cap[l]);
    }
    const unsigned long long leaf_cap = cap[nlev - 1];
    const unsigned long long atom_cap =
        (npix * (unsigned long long)P.cap_num + P.cap_den - 1) / P.cap_den + leaf_cap;

    const size_t out_off = (sizeof(PlaneDesc) * n_planes + 15) & ~(size_t)15;
    const size_t call_bytes = out_off + sizeof(OrderOut);
    if ((rc = c->planes.reserve(call_bytes))) return rc;
    if (!dev_in && (rc = c->staging.reserve(staged))) return rc;
    if ((rc = c->queues.reserve(sizeof(QueueEntry) * qoff[nlev]))) return rc;
    if ((rc = c->Y.reserve(sizeof(__nv_bfloat16) * ymax))) return rc;
    if ((rc = c->e0.reserve(sizeof(uint32_t) * emax))) return rc;
    if (fp8) {
        if ((rc = c->Y8.reserve(y8max))) return rc;
        if ((rc = c->inv_sl.reserve(sizeof(float) * emax))) return rc;
    }
    if ((rc = c->c0.reserve(sizeof(float2) * cmax))) return rc;
    if (resc) {
        unsigned long long rmax = 0, rcap = 0;
        for (int l = 0; l < nlev; ++l)
            if (corr_sepbf_available(P.max_block >> l)) {
                rmax = std::max(rmax, cap[l] * dicts[l]->d.M);
                rcap = std::max(rcap, cap[l]);
            }
        if (rmax) {
            if ((rc = c->ebound.reserve(sizeof(float) * rmax))) return rc;
            if ((rc = c->mu_buf.reserve(rcap))) return rc;
            if ((rc = c->fbq.reserve(sizeof(QueueEntry) * rcap))) return rc;
        }
    }
    // the pursuit kernels emit into the workspace; the ordering pass writes
    // the outputs, allocated per call from the stream-ordered pool at their
    // worst-case size
    const int zbits = 2 * (ilog2(P.max_block) - ilog2(P.min_block));
    const unsigned long long n_cells = roots << zbits;
    if ((rc = c->leaves_ws.reserve(sizeof(LeafRec) * leaf_cap))) return rc;
    if ((rc = c->atoms_ws.reserve(sizeof(AtomRec) * atom_cap))) return rc;
    if ((rc = c->lo_ws.reserve(sizeof(float) * atom_cap))) return rc;
    if ((rc = c->cells.reserve(sizeof(uint32_t) * n_cells))) return rc;
    if ((rc = c->perm.reserve(sizeof(uint32_t) * leaf_cap))) return rc;
    if ((rc = c->new_off.reserve(sizeof(uint32_t) * leaf_cap))) return rc;
    if ((rc = c->atom_leaf.reserve(sizeof(uint32_t) * atom_cap))) return rc;
    const unsigned long long status_words = order_status_words(n_cells, leaf_cap);
    if ((rc = c->order_status.reserve(sizeof(unsigned long long) * status_words))) return rc;
    auto code = std::make_unique<aqmp_code>();
    code->device = c->device;
    CK(cudaMallocFromPoolAsync((void **)&code->leaves, sizeof(LeafRec) * std::max<unsigned long long>(1, leaf_cap),
                               c->out_pool, st));
    CK(cudaMallocFromPoolAsync((void **)&code->atoms, sizeof(AtomRec) * std::max<unsigned long long>(1, atom_cap),
                               c->out_pool, st));
    CK(cudaMallocFromPoolAsync((void **)&code->alpha_lo, sizeof(float) * std::max<unsigned long long>(1, atom_cap),
                               c->out_pool, st));
    if ((rc = c->counters.reserve(sizeof(Counters)))) return rc;
    // OMP at sides 32 and 64: a packed Cholesky factor per resident CTA
    unsigned long long omp_doubles = 0;
    if (omp)
        for (int l = 0; l < nlev; ++l) {
            const int b = P.max_block >> l;
            if (b < 32) continue;
            const int kb = (int)std::max<long long>(1, (long long)b * b * P.cap_num / P.cap_den);
            omp_doubles = std::max(omp_doubles, omp_cta_workspace_doubles(kb, c->num_sms));
        }
    if (omp_doubles && (rc = c->omp_L.reserve(sizeof(double) * omp_doubles))) return rc;

    // plane descriptors (and host pixels copied in)
    std::vector<PlaneDesc> pd(n_planes);
    unsigned long long soff = 0, roff = 0;
    for (int i = 0; i < n_planes; ++i) {
        const aqmp_plane &pl = planes[i];
        PlaneDesc &d = pd[i];
        if (dev_in) {
            d.pix = pl.pixels;
            d.pitch = pl.pitch;
        } else {
            uint8_t *dst = (uint8_t *)c->staging.p + soff;
            // one linear copy for a contiguous plane (faster than the strided form)
            if (pl.pitch == pl.width)
                CK(cudaMemcpyAsync(dst, pl.pixels, (size_t)pl.height * pl.width, cudaMemcpyHostToDevice, st));
            else
                CK(cudaMemcpy2DAsync(dst, pl.width, pl.pixels, pl.pitch, pl.width, pl.height, cudaMemcpyHostToDevice,
                                     st));
            d.pix = dst;
            d.pitch = pl.width;
            soff += (unsigned long long)pl.height * pl.width;
        }
        d.h = pl.height;
        d.w = pl.width;
        d.tol = pl.rmse_tol < 0.0f ? P.rmse_tol : pl.rmse_tol;
        d.root_off = (unsigned)roff;
        d.roots_x = (unsigned)(pl.width / P.max_block);
        d.pad = 0;
        roff += (unsigned long long)(pl.height / P.max_block) * (pl.width / P.max_block);
    }
    if (c->host_call_cap < call_bytes) {
        if (c->host_call) cudaFreeHost(c->host_call);
        c->host_call = nullptr;
        c->host_call_cap = 0;
        g_ws_generation.fetch_add(1);
        CK(cudaMallocHost((void **)&c->host_call, std::max<size_t>(call_bytes, 4096)));
        c->host_call_cap = std::max<size_t>(call_bytes, 4096);
    }
    std::memcpy(c->host_call, pd.data(), sizeof(PlaneDesc) * n_planes);
    const OrderOut outs{code->leaves, code->atoms, code->alpha_lo};
    std::memcpy(c->host_call + out_off, &outs, sizeof outs);
    Counters *ctr = (Counters *)c->counters.p;
    const bool exact = P.precision == AQMP_PREC_EXACT || resc;     // double-float certified pursuit

    // A configuration whose kernel choices are settled is captured as a CUDA
    // graph on its second call and replayed from then on: everything from
    // the upload of this block to the read-back of the counters (the block
    // carries what changes between calls: plane addresses, tolerances and
    // output arrays).  AQMP_GRAPHS=0 in the environment turns this off.
    auto settled = [&]() {
        if (!tune) return true;
        for (int l = 0; l < nlev; ++l) {
            const int b = P.max_block >> l;
            if (!simt && !bf16 && !fp8 && !(resc && corr_sepbf_available(b)) && corr_sep_tc_available(b, dicts[l]->d.nf) &&
                c->tuner.slot(Tuner::CORR, b, P.dict_id, P.precision, cap[l]).chosen < 0)
                return false;
            if (!alt_threads && !omp && mp_has_variant(b, dicts[l]->d.nf) &&
                c->tuner.slot(Tuner::MP, b, P.dict_id, P.precision, cap[l]).chosen < 0)
                return false;
        }
        return true;
    };
    std::vector<long long> key{n_planes, P.cap_num, P.cap_den, P.min_block, P.max_block, P.dict_id, P.precision,
                               (long long)(P.flags & ~AQMP_FLAG_INPUT_DEVICE), dev_in ? 1 : 0, g_prof.on ? 1 : 0,
                               g_prof.on ? (long long)std::hash<std::string>{}(g_prof.filter) : 0};
    for (int i = 0; i < n_planes; ++i) {
        key.push_back(planes[i].height);
        key.push_back(planes[i].width);
    }
    static const bool graphs_on = [] {
        const char *v = std::getenv("AQMP_GRAPHS");
        return !(v && v[0] == '0');
    }();

    auto body = [&](cudaStream_t st) -> int {
    CK(cudaMemcpyAsync(c->planes.p, c->host_call, call_bytes, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), st));
    CK(cudaMemsetAsync(c->cells.p, 0, sizeof(uint32_t) * n_cells, st));
    CK(cudaMemsetAsync(c->order_status.p, 0, sizeof(unsigned long long) * status_words, st));
    const CellMap cells{(uint32_t *)c->cells.p, n_cells, P.max_block, P.min_block, zbits};
    QueueEntry *q = (QueueEntry *)c->queues.p;
    CK(launch_seed_roots((const PlaneDesc *)c->planes.p, n_planes, P.max_block, (unsigned)roots, q,
                         &ctr->queue_count[0], st));

    std::vector<CUtensorMap> ymaps(nlev), ysmaps(nlev);
    for (int l = 0; l < nlev; ++l) {
        const int b = P.max_block >> l;
        const DictDev &d = dicts[l]->d;
        LevelArgs lv{};
        lv.b = b;
        lv.n = d.n;
        lv.M = d.M;
        lv.Mpad = d.Mpad;
        lv.Kpad = d.Kpad;
        lv.k = (int)std::max<long long>(1, (long long)d.n * P.cap_num / P.cap_den);
        lv.level = l;
        lv.is_last = (l == nlev - 1);
        lv.queue = q + qoff[l];
        lv.count = &ctr->queue_count[l];
        lv.capacity = (unsigned)cap[l];
        lv.next_queue = lv.is_last ? nullptr : q + qoff[l + 1];
        lv.next_count = &ctr->queue_count[l + 1];
        lv.next_capacity = lv.is_last ? 0u : (unsigned)cap[l + 1];

        GatherArgs ga{b, d.n, d.Kpad, lv.queue, lv.count, lv.capacity, (const PlaneDesc *)c->planes.p,
                      (__nv_bfloat16 *)c->Y.p, (uint32_t *)c->e0.p, fp8 ? (uint8_t *)c->Y8.p : nullptr,
                      fp8 ? (float *)c->inv_sl.p : nullptr};
        const bool resc_l = resc && corr_sepbf_available(b);
        if (resc_l) ga.mu = (uint8_t *)c->mu_buf.p;
        CK(g_prof.run(kname("gather", b), st, [&] { return launch_gather(ga, c->num_sms, st); }));

        CorrArgs ca{};
        ca.d = &d;
        ca.Y = (const __nv_bfloat16 *)c->Y.p;
        ca.count = lv.count;
        ca.fixed_count = 0;
        ca.capacity = lv.capacity;
        ca.c0 = (float2 *)c->c0.p;
        ca.ctr = ctr;
        if (fp8) {
            if ((rc = encode_u8_map(&ymaps[l], c->Y8.p, cap[l], kpad_fp8(d.n), 64))) return rc;
        } else if ((rc = encode_bf16_map(&ymaps[l], c->Y.p, cap[l], d.Kpad, 64))) {
            return rc;
        }
        ca.tmap_Y = &ymaps[l];
        if (!fp8 && !bf16 && corr_sep_tc_available(b, d.nf)) {
            if ((rc = encode_bf16_map(&ysmaps[l], c->Y.p, cap[l] * (unsigned long long)b, b, b))) return rc;
            ca.tmap_Ysep = &ysmaps[l];
        }
        // exact correlation with the separable fixed-point dictionary: where
        // a tensor-core kernel for the side exists, the DCT-II family there
        // and the Haar family on the SIMT pipes, else (and with
        // AQMP_FLAG_SIMT_GEMM) all on the integer SIMT pipes; the two give
        // the same bits, so the autotuner may time both
        auto corr_tc = [&] { return corr_sep_hybrid(ca, b, st); };
        auto corr_simt = [&] {
            return g_prof.run(kname("corr_sep", b), st, [&] { return launch_corr_sep_simt(ca, st); });
        };
        const bool tc_ok = corr_sep_tc_available(b, d.nf);
        if (resc_l) {
            ca.mu = (const uint8_t *)c->mu_buf.p;
            ca.ebound = (float *)c->ebound.p;
            CK(g_prof.run(kname("corr_sepbf", b), st, [&] { return launch_corr_sepbf(ca, st); }));
        } else if (bf16) {
            CK(g_prof.run(kname("corr_bf16", b), st, [&] { return launch_corr_tc_bf16(ca, st); }));
        } else if (fp8) {
            CK(g_prof.run(kname("corr_fp8", b), st,
                          [&] { return launch_corr_tc_fp8(ca, (const float *)c->inv_sl.p, st); }));
        } else if (simt || !tc_ok) {
            CK(corr_simt());
        } else if (!tune) {
            CK(corr_tc());
        } else {
            Tuner::Slot &ts = c->tuner.slot(Tuner::CORR, b, P.dict_id, P.precision, cap[l]);
            if (ts.chosen >= 0) {
                CK(ts.chosen ? corr_simt() : corr_tc());
            } else {
                for (int rep = 0; rep < Tuner::kSamples; ++rep) {
                    CK(c->tuner.timed(ts, 0, st, corr_tc));
                    CK(c->tuner.timed(ts, 1, st, corr_simt));
                }
            }
        }

        MPArgs ma{};
        ma.lv = lv;
        ma.c0 = (const float2 *)c->c0.p;
        ma.e0 = (const uint32_t *)c->e0.p;
        ma.planes = (const PlaneDesc *)c->planes.p;
        ma.W = d.W;
        ma.WT = d.WT;
        ma.leaves = (LeafRec *)c->leaves_ws.p;
        ma.leaf_cap = leaf_cap;
        ma.atoms = (AtomRec *)c->atoms_ws.p;
        ma.alpha_lo = (float *)c->lo_ws.p;
        ma.atom_leaf = (uint32_t *)c->atom_leaf.p;
        ma.atom_cap = atom_cap;
        ma.cells = cells;
        ma.ctr = ctr;
        ma.omp_L = (double *)c->omp_L.p;
        ma.omp_slots = c->num_sms;
        ma.omp_L_doubles = omp_doubles;
        ma.fam0 = d.fam0;
        if (resc_l) {
            ma.ebound = (const float *)c->ebound.p;
            ma.Yc = (const __nv_bfloat16 *)c->Y.p;
            ma.Kpad = d.Kpad;
            ma.mu = (const uint8_t *)c->mu_buf.p;
            ma.Bs = d.Bs;
            ma.Rs = d.Rs;
            ma.fb_queue = (QueueEntry *)c->fbq.p;
            ma.fb_count = &ctr->fb_count[l];
            ma.fb_capacity = lv.capacity;
        }
        auto mp = [&](int v) {
            return g_prof.run(kname(resc_l ? "mp_resc" : exact ? "mp" : "mp_fp32", b), st,
                              [&] { return launch_mp(ma, d.nf, exact, v, c->num_sms, st); });
        };
        if (omp) {
            CK(g_prof.run(kname("omp", b), st, [&] { return launch_omp(ma, d.nf, c->num_sms, st); }));
        } else if (alt_threads || !tune || !mp_has_variant(b, d.nf)) {
            CK(mp(alt_threads ? 1 : 0));
        } else {
            Tuner::Slot &ts = c->tuner.slot(Tuner::MP, b, P.dict_id, P.precision, cap[l]);
            if (ts.chosen >= 0) {
                CK(mp(ts.chosen));
            } else {
                const int v = Tuner::next(ts);
                CK(c->tuner.timed(ts, v, st, [&] { return mp(v); }));
            }
        }
        if (resc_l) {
            // the leaves the rescore handed back, through the exact form: the
            // gather centred on 128, the exact correlation, the exact pursuit
            // (its own leaf counter), children and emission as for any leaf
            GatherArgs gf = ga;
            gf.queue = (const QueueEntry *)c->fbq.p;
            gf.count = &ctr->fb_count[l];
            gf.mu = nullptr;
            CK(g_prof.run(kname("gather_fb", b), st, [&] { return launch_gather(gf, c->num_sms, st); }));
            CorrArgs cf = ca;
            cf.count = &ctr->fb_count[l];
            cf.mu = nullptr;
            cf.ebound = nullptr;
            CK(g_prof.run(kname("corr_fb", b), st, [&] { return launch_corr_sep_tc(cf, st); }));
            MPArgs mf = ma;
            mf.lv.queue = (const QueueEntry *)c->fbq.p;
            mf.lv.count = &ctr->fb_count[l];
            mf.work = &ctr->work_fb[l];
            mf.ebound = nullptr;
            CK(g_prof.run(kname("mp_fb", b), st, [&] { return launch_mp(mf, d.nf, true, 0, c->num_sms, st); }));
        }
    }

    // canonical order of the output list: plane, root (raster), depth-first
    OrderArgs oa{};
    oa.cells = cells;
    oa.leaves_in = (const LeafRec *)c->leaves_ws.p;
    oa.atoms_in = (const AtomRec *)c->atoms_ws.p;
    oa.lo_in = (const float *)c->lo_ws.p;
    oa.atom_leaf = (const uint32_t *)c->atom_leaf.p;
    oa.n_leaves = &ctr->n_leaves;
    oa.n_atoms = &ctr->n_atoms;
    oa.new_off = (uint32_t *)c->new_off.p;
    oa.leaf_cap = leaf_cap;
    oa.atom_cap = atom_cap;
    oa.perm = (uint32_t *)c->perm.p;
    oa.status = (unsigned long long *)c->order_status.p;
    oa.out = (const OrderOut *)((unsigned char *)c->planes.p + out_off);
    oa.ctr = ctr;
    oa.limit_ns = 2000000000ull;
    CK(g_prof.run("order_rank", st, [&] { return launch_order_phase(oa, 0, c->num_sms, st); }));
    CK(g_prof.run("order_offsets", st, [&] { return launch_order_phase(oa, 1, c->num_sms, st); }));
    CK(g_prof.run("order_copy", st, [&] { return launch_order_phase(oa, 2, c->num_sms, st); }));

    CK(cudaMemcpyAsync(c->host_ctr, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    return AQMP_OK;
    };

    // a graph runs on the library's own stream, ordered after the caller's
    // prior work and before its later work
    auto replay = [&](Ctx::Graph &gr) -> int {
        CK(cudaEventRecord(c->graph_in, st));
        CK(cudaStreamWaitEvent(c->graph_stream, c->graph_in, 0));
        CK(cudaEventRecord(c->dev_t0, c->graph_stream));
        CK(cudaGraphLaunch(gr.exec, c->graph_stream));
        CK(cudaEventRecord(c->dev_t1, c->graph_stream));
        CK(cudaEventRecord(c->graph_out, c->graph_stream));
        CK(cudaStreamWaitEvent(st, c->graph_out, 0));
        if (!gr.prof.empty()) {
            std::lock_guard<std::mutex> pl(g_prof.mu);
            for (const auto &p : gr.prof) g_prof.pending.push_back(p);
        }
        return AQMP_OK;
    };
    if (!c->dev_t0) {
        CK(cudaEventCreate(&c->dev_t0));
        CK(cudaEventCreate(&c->dev_t1));
    }
    c->last_device_ms = -1.0f;
    auto git = c->graphs.find(key);
    if (git != c->graphs.end() && git->second.generation != g_ws_generation.load()) {
        c->drop_graphs();
        git = c->graphs.end();
    }
    if (graphs_on && git != c->graphs.end()) {
        if ((rc = replay(git->second))) return rc;
    } else {
        if (c->seen.size() > 1024) c->seen.clear();
        int &runs = c->seen[key];
        bool done = false;
        if (graphs_on && runs >= 1 && settled()) {
            runs = -1;                            // unless the capture below succeeds
            if (c->graphs.size() >= 32) c->drop_graphs();
            if (!c->graph_stream) {
                CK(cudaStreamCreateWithFlags(&c->graph_stream, cudaStreamNonBlocking));
                CK(cudaEventCreateWithFlags(&c->graph_in, cudaEventDisableTiming));
                CK(cudaEventCreateWithFlags(&c->graph_out, cudaEventDisableTiming));
            }
            Ctx::Graph gr;
            gr.generation = g_ws_generation.load();
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(c->graph_stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
                Profiler::capture_to = &gr.prof;
                const int brc = body(c->graph_stream);
                Profiler::capture_to = nullptr;
                const cudaError_t ec = cudaStreamEndCapture(c->graph_stream, &graph);
                if (brc == AQMP_OK && ec == cudaSuccess && graph &&
                    cudaGraphInstantiate(&gr.exec, graph, 0) == cudaSuccess) {
                    cudaGraphDestroy(graph);
                    auto &slot = c->graphs[key];
                    slot = std::move(gr);
                    if ((rc = replay(slot))) return rc;
                    runs = 1;
                    done = true;
                } else {
                    if (graph) cudaGraphDestroy(graph);
                    for (auto &p : gr.prof) {
                        cudaEventDestroy(p.a);
                        cudaEventDestroy(p.b);
                    }
                }
            }
            cudaGetLastError();
        }
        if (!done) {
            CK(cudaEventRecord(c->dev_t0, st));
            if ((rc = body(st))) return rc;
            CK(cudaEventRecord(c->dev_t1, st));
            if (runs >= 0) ++runs;
        }
    }
    CK(cudaStreamSynchronize(st));
    {
        float ms = -1.0f;
        if (cudaEventElapsedTime(&ms, c->dev_t0, c->dev_t1) == cudaSuccess) c->last_device_ms = ms;
        cudaGetLastError();
    }
    {
        std::lock_guard<std::mutex> pl(g_prof.mu);
        g_prof.resolve();
    }
    c->tuner.resolve();
    const Counters &h = *c->host_ctr;
    if (h.error == kDevErrQueueOverflow) return fail(AQMP_E_QUEUE_OVERFLOW, "device queue overflow (site %u)", h.error_info);
    if (h.error == kDevErrTimeout) return fail(AQMP_E_TIMEOUT, "device wait timed out (site %u)", h.error_info);
    if (h.error) return fail(AQMP_E_CUDA, "device error %u (%u)", h.error, h.error_info);

    code->dict_id = P.dict_id;
    code->min_block = P.min_block;
    code->max_block = P.max_block;
    for (int i = 0; i < n_planes; ++i) code->shapes.emplace_back(planes[i].height, planes[i].width);
    code->n_leaves = h.n_leaves;
    code->n_atoms = h.n_atoms;
    aqmp_stats &s = code->stats;
    s.n_leaves = h.n_leaves;
    s.n_atoms = h.n_atoms;
    s.near_tie_leaves = h.near_tie_leaves;
    for (int l = 0; l < nlev && l < 8; ++l) {
        s.attempts_per_level[l] = h.attempts[l];
        s.iterations_per_level[l] = h.iterations[l];
        s.window_steps_per_level[l] = h.window_steps[l];
        s.max_leaf_steps_per_level[l] = h.max_steps[l];
        s.attempts += h.attempts[l];
        s.atom_iterations += h.iterations[l];
        s.rescored_atoms += h.rescored[l];
        s.rescore_rounds += h.resc_rounds[l];
        s.fallback_leaves += h.fallbacks[l];
    }
    *out = code.release();
    return AQMP_OK;
}

int aqmp_encode(const aqmp_params *params, const uint8_t *pixels, int channels, int h, int w, size_t pitch,
                void *stream, aqmp_code **out) {
    if (!pixels || channels <= 0) return fail(AQMP_E_ARG, "no pixels");
    std::vector<aqmp_plane> pl(channels);
    for (int c = 0; c < channels; ++c) {
        pl[c].pixels = pixels + (size_t)c * h * pitch;
        pl[c].height = h;
        pl[c].width = w;
        pl[c].pitch = (int64_t)pitch;
        pl[c].rmse_tol = -1.0f;
    }
    return aqmp_encode_planes(params, pl.data(), channels, stream, out);
}

int aqmp_encode_batch(const aqmp_params *params, int n_images, const uint8_t *const *images, const int *channels,
                      const int *h, const int *w, const size_t *pitch, void *stream, aqmp_code **out) {
    if (n_images <= 0 || !images || !channels || !h || !w || !pitch) return fail(AQMP_E_ARG, "bad batch arguments");
    std::vector<aqmp_plane> pl;
    for (int i = 0; i < n_images; ++i) {
        if (!images[i] || channels[i] <= 0) return fail(AQMP_E_ARG, "image %d: no pixels", i);
        for (int c = 0; c < channels[i]; ++c) {
            aqmp_plane p{};
            p.pixels = images[i] + (size_t)c * h[i] * pitch[i];
            p.height = h[i];
            p.width = w[i];
            p.pitch = (int64_t)pitch[i];
            p.rmse_tol = -1.0f;
            pl.push_back(p);
        }
    }
    return aqmp_encode_planes(params, pl.data(), (int)pl.size(), stream, out);
}

int aqmp_code_stats(const aqmp_code *code, aqmp_stats *stats) {
    if (!code || !stats) return fail(AQMP_E_ARG, "NULL argument");
    *stats = code->stats;
    return AQMP_OK;
}

int aqmp_code_copy(const aqmp_code *code, aqmp_leaf *leaves, aqmp_atom *atoms, float *alpha_lo) {
    if (!code || (!leaves && code->n_leaves) || (!atoms && code->n_atoms)) return fail(AQMP_E_ARG, "NULL argument");
    // the device arrays are already in canonical order (written so by the
    // encode); the three transfers are queued together and waited for once
    // (into page-locked buffers they overlap; pageable ones are staged)
    cudaStream_t st = cudaStreamLegacy;
    if (code->n_leaves)
        CK(cudaMemcpyAsync(leaves, code->leaves, sizeof(LeafRec) * code->n_leaves, cudaMemcpyDeviceToHost, st));
    if (code->n_atoms) {
        CK(cudaMemcpyAsync(atoms, code->atoms, sizeof(AtomRec) * code->n_atoms, cudaMemcpyDeviceToHost, st));
        if (alpha_lo)
            CK(cudaMemcpyAsync(alpha_lo, code->alpha_lo, sizeof(float) * code->n_atoms, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    return AQMP_OK;
}

int aqmp_decode(const aqmp_code *code, int plane, float *out, int64_t out_pitch, int out_is_device, void *stream) {
    g_last_error.clear();
    if (!code || !out || plane < 0 || plane >= (int)code->shapes.size()) return fail(AQMP_E_ARG, "bad argument");
    const int h = code->shapes[plane].first, w = code->shapes[plane].second;
    if (out_pitch < w) return fail(AQMP_E_ARG, "out_pitch below width");
    Ctx *c;
    int rc;
    if ((rc = get_ctx(&c))) return rc;
    std::lock_guard<std::mutex> lock(c->mu);
    cudaStream_t st = (cudaStream_t)stream;
    DecodeArgs a{};
    a.leaves = code->leaves;
    a.n_leaves = code->n_leaves;
    a.atoms = code->atoms;
    a.plane = (uint32_t)plane;
    a.nf = num_families(code->dict_id);
    a.single_family = 0;
    for (int b = code->min_block; b <= code->max_block; b *= 2) {
        Dict *d;
        if ((rc = get_dict(c, b, code->dict_id, st, &d, false))) return rc;
        a.basis[ilog2(b)] = d->d.basis;
    }
    float *dst = out;
    long long pitch = out_pitch;
    void *tmp = nullptr;
    if (!out_is_device) {
        CK(cudaMalloc(&tmp, sizeof(float) * (size_t)h * w));
        dst = (float *)tmp;
        pitch = w;
    }
    a.out = dst;
    a.out_pitch = pitch;
    cudaError_t e = g_prof.run(kname("decode", code->max_block), st, [&] { return launch_decode(a, c->num_sms, st); });
    if (e == cudaSuccess && !out_is_device)
        e = cudaMemcpy2DAsync(out, sizeof(float) * out_pitch, dst, sizeof(float) * w, sizeof(float) * w, h,
                              cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> pl(g_prof.mu);
        g_prof.resolve();
    }
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return fail(AQMP_E_CUDA, "decode: %s", cudaGetErrorString(e));
    return AQMP_OK;
}

void aqmp_code_free(aqmp_code *code) { delete code; }

int aqmp_code_device(const aqmp_code *code, const aqmp_leaf **leaves, const aqmp_atom **atoms, uint64_t *n_leaves,
                     uint64_t *n_atoms) {
    if (!code || !leaves || !atoms || !n_leaves || !n_atoms) return fail(AQMP_E_ARG, "NULL argument");
    *leaves = reinterpret_cast<const aqmp_leaf *>(code->leaves);
    *atoms = reinterpret_cast<const aqmp_atom *>(code->atoms);
    *n_leaves = code->n_leaves;
    *n_atoms = code->n_atoms;
    return AQMP_OK;
}

// Basis tables of every side a code uses, for the synthesis kernels.
static int code_bases(Ctx *c, const aqmp_code *code, cudaStream_t st, DecodeArgs *a) {
    *a = DecodeArgs{};
    a->nf = num_families(code->dict_id);
    a->single_family = 0;
    for (int b = code->min_block; b <= code->max_block; b *= 2) {
        Dict *d;
        int rc = get_dict(c, b, code->dict_id, st, &d, false);
        if (rc) return rc;
        a->basis[ilog2(b)] = d->d.basis;
    }
    return AQMP_OK;
}

int aqmp_synth_forward(const aqmp_code *code, int plane, const float *alpha, float *out, int64_t out_pitch,
                       void *stream) {
    g_last_error.clear();
    if (!code || !alpha || !out || plane < 0 || plane >= (int)code->shapes.size()) return fail(AQMP_E_ARG, "bad argument");
    if (out_pitch < code->shapes[plane].second) return fail(AQMP_E_ARG, "out_pitch below width");
    Ctx *c;
    int rc;
    if ((rc = get_ctx(&c))) return rc;
    std::lock_guard<std::mutex> lock(c->mu);
    cudaStream_t st = (cudaStream_t)stream;
    DecodeArgs bases;
    if ((rc = code_bases(c, code, st, &bases))) return rc;
    CK(g_prof.run(kname("synth_fwd", code->max_block), st, [&] {
        return launch_synth_forward(code->leaves, code->n_leaves, code->atoms, alpha, (uint32_t)plane, out,
                                    out_pitch, bases, c->num_sms, st);
    }));
    return AQMP_OK;
}

int aqmp_synth_backward(const aqmp_code *code, int plane, const float *grad_out, int64_t pitch, float *grad_alpha,
                        void *stream) {
    g_last_error.clear();
    if (!code || !grad_out || !grad_alpha || plane < 0 || plane >= (int)code->shapes.size())
        return fail(AQMP_E_ARG, "bad argument");
    if (pitch < code->shapes[plane].second) return fail(AQMP_E_ARG, "pitch below width");
    Ctx *c;
    int rc;
    if ((rc = get_ctx(&c))) return rc;
    std::lock_guard<std::mutex> lock(c->mu);
    cudaStream_t st = (cudaStream_t)stream;
    DecodeArgs bases;
    if ((rc = code_bases(c, code, st, &bases))) return rc;
    CK(g_prof.run(kname("synth_bwd", code->max_block), st, [&] {
        return launch_synth_backward(code->leaves, code->n_leaves, code->atoms, (uint32_t)plane, grad_out, pitch,
                                     grad_alpha, bases, code->max_block, c->num_sms, st);
    }));
    return AQMP_OK;
}

int aqmp_ssim(const float *x, const float *y, int h, int w, int64_t pitch, double *ssim, float *grad_y,
              double grad_scale, void *stream) {
    g_last_error.clear();
    if (!x || !y || !ssim || h < 11 || w < 11 || pitch < w) return fail(AQMP_E_ARG, "bad argument");
    Ctx *c;
    int rc;
    if ((rc = get_ctx(&c))) return rc;
    std::lock_guard<std::mutex> lock(c->mu);
    cudaStream_t st = (cudaStream_t)stream;
    if (!c->gauss_ready) {
        CK(upload_gauss11(st));
        c->gauss_ready = true;
    }
    const size_t hw = (size_t)h * (w - 10), win = (size_t)(h - 10) * (w - 10);
    if ((rc = c->ssim_ws.reserve(sizeof(double) * (5 * hw + 3 * win + 3 * hw)))) return rc;
    double *H = (double *)c->ssim_ws.p, *P = H + 5 * hw, *V = P + 3 * win;
    CK(cudaMemsetAsync(ssim, 0, sizeof(double), st));
    CK(g_prof.run(grad_y ? "ssim_fwd_bwd" : "ssim_fwd", st,
                  [&] { return launch_ssim(x, y, h, w, pitch, H, P, V, ssim, grad_y, grad_scale, c->num_sms, st); }));
    return AQMP_OK;
}

int aqmp_selftest_wait(int limit_ms, void *stream) {
    g_last_error.clear();
    if (limit_ms < 1 || limit_ms > 5000) return fail(AQMP_E_ARG, "limit_ms must be in [1, 5000]");
    Ctx *c;
    int rc;
    if ((rc = get_ctx(&c))) return rc;
    std::lock_guard<std::mutex> lock(c->mu);
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = c->counters.reserve(sizeof(Counters)))) return rc;
    Counters *ctr = (Counters *)c->counters.p;
    CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), st));
    CK(launch_wait_selftest(ctr, (unsigned long long)limit_ms * 1000000ull, st));
    CK(cudaMemcpyAsync(c->host_ctr, ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (c->host_ctr->error == kDevErrTimeout)
        return fail(AQMP_E_TIMEOUT, "bounded device wait gave up after %d ms (as intended)", limit_ms);
    return AQMP_OK;
}

int aqmp_selftest_round(const int64_t *words, int64_t n, float *out, void *stream) {
    g_last_error.clear();
    if (n < 0 || n > 0x7fffffffLL || (n > 0 && (!words || !out))) return fail(AQMP_E_ARG, "bad arguments");
    if (n == 0) return AQMP_OK;
    if (((uintptr_t)words & 7) != 0 || ((uintptr_t)out & 7) != 0)
        return fail(AQMP_E_ARG, "words and out must be 8-byte aligned");
    Ctx *c;
    int rc;
    if ((rc = get_ctx(&c))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    CK(launch_round_selftest((const long long *)words, (long long)n, (float2 *)out, st));
    CK(cudaStreamSynchronize(st));
    return AQMP_OK;
}

int aqmp_profile_enable(int on) {
    std::lock_guard<std::mutex> g(g_prof.mu);
    const int prev = g_prof.on ? 1 : 0;
    g_prof.on = on != 0;
    return prev;
}

void aqmp_profile_reset(void) {
    std::lock_guard<std::mutex> g(g_prof.mu);
    g_prof.totals.clear();
}

int aqmp_profile_filter(const char *prefix) {
    std::lock_guard<std::mutex> g(g_prof.mu);
    g_prof.filter = prefix ? prefix : "";
    return AQMP_OK;
}

int aqmp_profile_read(aqmp_kernel_time *out, int max, int *n) {
    if (!n || (max > 0 && !out)) return fail(AQMP_E_ARG, "NULL argument");
    std::lock_guard<std::mutex> g(g_prof.mu);
    int i = 0;
    for (auto &kv : g_prof.totals) {
        if (i < max) {
            std::memset(&out[i], 0, sizeof(aqmp_kernel_time));
            std::strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
            out[i].launches = kv.second.first;
            out[i].total_ms = kv.second.second;
        }
        ++i;
    }
    *n = std::min(i, std::max(max, 0));
    return AQMP_OK;
}

int aqmp_correlate_bf16x2(int b, int dict_id, const uint8_t *blocks, int64_t L, float *corr, float *bound,
                          void *stream) {
    g_last_error.clear();
    if (!corr_sepbf_available(b)) return fail(AQMP_E_UNSUPPORTED, "the BF16 form with rescore serves side 64 only");
    if (dict_id < 0 || dict_id > 2) return fail(AQMP_E_DICT, "unknown dictionary id %d", dict_id);
    if (L < 0 || (L > 0 && (!blocks || !corr || !bound))) return fail(AQMP_E_ARG, "bad pointers");
    if (L == 0) return AQMP_OK;
    if (L > 0x7fffffffLL) return fail(AQMP_E_UNSUPPORTED, "too many blocks");
    Ctx *c;
    int rc;
    if ((rc = get_ctx(&c))) return rc;
    std::lock_guard<std::mutex> lock(c->mu);
    cudaStream_t st = (cudaStream_t)stream;
    Dict *D;
    if ((rc = get_dict(c, b, dict_id, st, &D, false))) return rc;
    const DictDev &d = D->d;
    if ((rc = c->Y.reserve(sizeof(__nv_bfloat16) * (size_t)L * d.Kpad))) return rc;
    if ((rc = c->mu_buf.reserve((size_t)L))) return rc;
    CUtensorMap ysm;
    if ((rc = encode_bf16_map(&ysm, c->Y.p, (unsigned long long)L * b, b, b))) return rc;
    CK(launch_gather_blocks(b, d.Kpad, blocks, L, (__nv_bfloat16 *)c->Y.p, nullptr, c->num_sms, st,
                            (uint8_t *)c->mu_buf.p));
    CorrArgs ca{};
    ca.d = &d;
    ca.Y = (const __nv_bfloat16 *)c->Y.p;
    ca.fixed_count = L;
    ca.capacity = (unsigned)L;
    ca.c0 = (float2 *)corr;
    ca.tmap_Ysep = &ysm;
    ca.mu = (const uint8_t *)c->mu_buf.p;
    ca.ebound = bound;
    const cudaError_t e = g_prof.run(kname("corr_sepbf", b), st, [&] { return launch_corr_sepbf(ca, st); });
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        return fail(AQMP_E_CUDA, "correlation kernel: %s", cudaGetErrorString(e));
    }
    CK(cudaStreamSynchronize(st));
    {
        std::lock_guard<std::mutex> pl(g_prof.mu);
        g_prof.resolve();
    }
    return AQMP_OK;
}

int aqmp_correlate(int b, int dict_id, const uint8_t *blocks, int64_t L, float *corr, int gemm, void *stream) {
    g_last_error.clear();
    if (!is_pow2(b) || b < 4 || b > kMaxSide) return fail(AQMP_E_ARG, "side must be a power of two in [4, %d]", kMaxSide);
    if (dict_id < 0 || dict_id > 2) return fail(AQMP_E_DICT, "unknown dictionary id %d", dict_id);
    if (L < 0 || (L > 0 && (!blocks || !corr))) return fail(AQMP_E_ARG, "bad pointers");
    if (gemm < 0 || gemm > 6)
        return fail(AQMP_E_ARG, "gemm must be 0 (separable, best kernel), 1 (separable SIMT), 2 (BF16 form), "
                                "3 (dense tensor cores), 4 (dense SIMT), 5 (FP8 form) or 6 (separable "
                                "tensor cores, every family)");
    if (gemm == 6 && !corr_sep_tc_available(b, 2))
        return fail(AQMP_E_UNSUPPORTED, "no separable tensor-core kernel for side %d", b);
    if (L == 0) return AQMP_OK;
    if (((uintptr_t)corr & 15) != 0) return fail(AQMP_E_ARG, "corr must be 16-byte aligned");
    if (L > 0x7fffffffLL) return fail(AQMP_E_UNSUPPORTED, "too many blocks");
    Ctx *c;
    int rc;
    if ((rc = get_ctx(&c))) return rc;
    std::lock_guard<std::mutex> lock(c->mu);
    cudaStream_t st = (cudaStream_t)stream;
    const bool dense = gemm == 3 || gemm == 4;
    Dict *D;
    if ((rc = get_dict(c, b, dict_id, st, &D, dense, gemm == 2, gemm == 5))) return rc;
    const DictDev &d = D->d;
    CUtensorMap ym, ysm;
    if (gemm == 5) {
        if ((rc = c->Y8.reserve((size_t)L * kpad_fp8(d.n)))) return rc;
        if ((rc = c->inv_sl.reserve(sizeof(float) * (size_t)L))) return rc;
        if ((rc = encode_u8_map(&ym, c->Y8.p, (unsigned long long)L, kpad_fp8(d.n), 64))) return rc;
        CK(launch_gather_blocks_fp8(b, blocks, L, (uint8_t *)c->Y8.p, (float *)c->inv_sl.p, c->num_sms, st));
    } else {
        if ((rc = c->Y.reserve(sizeof(__nv_bfloat16) * (size_t)L * d.Kpad))) return rc;
        if (gemm != 1 && gemm != 4) {
            if ((rc = encode_bf16_map(&ym, c->Y.p, (unsigned long long)L, d.Kpad, 64))) return rc;
        }
        if ((gemm == 0 || gemm == 6) && corr_sep_tc_available(b, d.nf)) {
            if ((rc = encode_bf16_map(&ysm, c->Y.p, (unsigned long long)L * b, b, b))) return rc;
        }
        CK(launch_gather_blocks(b, d.Kpad, blocks, L, (__nv_bfloat16 *)c->Y.p, nullptr, c->num_sms, st));
    }
    CorrArgs ca{};
    ca.d = &d;
    ca.Y = (const __nv_bfloat16 *)c->Y.p;
    ca.count = nullptr;
    ca.fixed_count = L;
    ca.capacity = (unsigned)L;
    ca.c0 = (float2 *)corr;
    ca.tmap_Y = &ym;
    ca.tmap_Ysep = &ysm;
    cudaError_t e = cudaSuccess;
    switch (gemm) {
        case 0:
            e = corr_sep_tc_available(b, d.nf)
                    ? corr_sep_hybrid(ca, b, st)
                    : g_prof.run(kname("corr_sep", b), st, [&] { return launch_corr_sep_simt(ca, st); });
            break;
        case 6: e = g_prof.run(kname("corr_septc", b), st, [&] { return launch_corr_sep_tc(ca, st); }); break;
        case 1: e = g_prof.run(kname("corr_sep", b), st, [&] { return launch_corr_sep_simt(ca, st); }); break;
        case 2: e = g_prof.run(kname("corr_bf16", b), st, [&] { return launch_corr_tc_bf16(ca, st); }); break;
        case 3: e = g_prof.run(kname("corr_tc", b), st, [&] { return launch_corr_tc(ca, st); }); break;
        case 4: e = g_prof.run(kname("corr_simt", b), st, [&] { return launch_corr_simt(ca, st); }); break;
        case 5:
            e = g_prof.run(kname("corr_fp8", b), st,
                           [&] { return launch_corr_tc_fp8(ca, (const float *)c->inv_sl.p, st); });
            break;
    }
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        return fail(AQMP_E_CUDA, "correlation kernel: %s", cudaGetErrorString(e));
    }
    CK(cudaStreamSynchronize(st));
    {
        std::lock_guard<std::mutex> pl(g_prof.mu);
        g_prof.resolve();
    }
    return AQMP_OK;
}

}  // extern "C"
