// noalloc.cu -- aqmp_correlate_noalloc: the initial-correlation entry point
// without any device allocation.
//
// Some callers cannot call cudaMalloc: hosts whose device memory belongs to
// another allocator that has to account for every byte (a caching allocator
// such as PyTorch's, or a fixed per-process budget in a shared service), and
// real-time loops that reserve all their memory when they start because an
// allocation can block or fail at run time.  For them this file keeps the
// scratch of the correlation -- the gathered, centred BF16 block vectors the
// tensor-core kernel reads -- together with the fixed-point dictionary tables
// of one block side and an error word, in file-scope __device__ arrays of
// fixed size.  Every GPU that loads the library holds these arrays (about
// 10.1 MB) until the process exits.
//
// Limits: block side 4, 8 or 16; at most kScratchBytes / (Kpad * 2) blocks per
// call (65536 blocks of side 4 or 8, 16384 of side 16).  Larger requests are
// rejected with AQMP_E_ARG; they never fall back to allocating.
//
// In host code the arrays' names are host-side stand-ins, not device
// addresses, so the first call on each device looks their device addresses up
// with cudaGetSymbolAddress (with that device current) and keeps them; that
// first call should come before any stream capture.  No call can be captured
// into a CUDA graph: every call waits for its stream and reads a status word
// back, so a call on a capturing stream returns AQMP_E_UNSUPPORTED without
// touching the stream.  Every call shares the arrays and they keep the
// previous call's contents: the table region is cleared before it is rebuilt,
// the error word at every call, and each call rewrites every scratch byte it
// reads.  Calls whose GPU work overlaps would race on the arrays; this entry
// point serialises its callers and synchronises the stream before returning
// (on an error too, once it has queued work), so calls made through it never
// overlap.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/aqmp.h"
#include "common.cuh"
#include "kernels.h"

using namespace aqmp;

namespace {

constexpr int kMaxSide = 16;
constexpr int kMaxAtoms = 2 * kMaxSide * kMaxSide;              // 512
constexpr int kMaxKpad = kMaxSide * kMaxSide;                   // 256
constexpr int kMaxMpad = kMaxAtoms;                             // multiple of 128
constexpr size_t kScratchBytes = size_t(8) << 20;               // gathered blocks

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];
__device__ __align__(256) __nv_bfloat16 g_limbs[kLimbs * kMaxMpad * kMaxKpad];
__device__ __align__(256) long long g_sums[2 * kMaxAtoms];
__device__ __align__(256) double g_basis[2 * kMaxSide * kMaxSide];
__device__ __align__(256) Counters g_counters;                  // error word of the kernels

struct Slot {
    void *scratch = nullptr, *limbs = nullptr, *sums = nullptr, *basis = nullptr, *counters = nullptr;
    int table_b = 0, table_dict = -1;
    int sms = 0;
    CUtensorMap limb_map;
};

std::mutex g_mu;
std::map<int, Slot> g_slots;

// Device addresses of the arrays on the current device (set-up, once per device).
int device_slot(Slot **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(AQMP_E_CUDA, "no CUDA device");
    auto it = g_slots.find(dev);
    if (it == g_slots.end()) {
        Slot s;
        int major = 0, minor = 0;
        if (cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
            return set_error(AQMP_E_CUDA, "cannot query the current device");
        if (major != 10 || minor != 3) return set_error(AQMP_E_CUDA, "this library is built for sm_103a only");
        if (cudaGetSymbolAddress(&s.scratch, g_scratch) != cudaSuccess ||
            cudaGetSymbolAddress(&s.limbs, g_limbs) != cudaSuccess ||
            cudaGetSymbolAddress(&s.sums, g_sums) != cudaSuccess ||
            cudaGetSymbolAddress(&s.basis, g_basis) != cudaSuccess ||
            cudaGetSymbolAddress(&s.counters, g_counters) != cudaSuccess)
            return set_error(AQMP_E_CUDA, "cudaGetSymbolAddress failed for the static scratch");
        it = g_slots.emplace(dev, s).first;
    }
    *out = &it->second;
    return AQMP_OK;
}

// Fixed-point digits and per-atom sums of one (side, dictionary), written
// into the static tables (same construction as the library's table builder:
// D_fix = round(D 2^48), 8 balanced base-64 digits, S_j = sum_v D_fix).
__global__ void static_tables_kernel(int b, int nf, int fam0, const double *basis, int Mpad, int Kpad,
                                     __nv_bfloat16 *limbs, long long *sums) {
    const int n = b * b, M = nf * n;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < M; j += warps) {
        const int fam = nf == 2 ? j / n : fam0;
        const int f = nf == 2 ? j - (j / n) * n : j;
        const int p = f % b, q = f / b;
        const double *B = basis + (size_t)fam * b * b;
        long long s = 0;
        for (int v = lane; v < n; v += 32) {
            const int m = v / b, i = v - m * b;
            const long long x = __double2ll_rn(B[p * b + i] * B[q * b + m] * 281474976710656.0);
            s += x;
            long long r = x;
            for (int d = kLimbs - 1; d >= 1; --d) {
                const long long dg = ((r + 32) & 63) - 32;
                limbs[((size_t)d * Mpad + j) * Kpad + v] = __float2bfloat16_rn((float)dg);
                r = (r - dg) >> kDigitBits;
            }
            limbs[(size_t)j * Kpad + v] = __float2bfloat16_rn((float)r);
        }
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) {
            const long long h = (s + (1ll << 23)) >> 24;
            sums[j] = h;
            sums[kMaxAtoms + j] = s - h * (1ll << 24);
        }
    }
}

}  // namespace

extern "C" int aqmp_correlate_noalloc(int b, int dict_id, const uint8_t *blocks, int64_t L, float *corr,
                                      void *stream) {
    set_error(AQMP_OK, "");
    if (b != 4 && b != 8 && b != 16)
        return set_error(AQMP_E_ARG, "aqmp_correlate_noalloc: block side must be 4, 8 or 16");
    if (dict_id < 0 || dict_id > 2) return set_error(AQMP_E_DICT, "unknown dictionary id");
    if (L < 0 || (L > 0 && (!blocks || !corr))) return set_error(AQMP_E_ARG, "bad pointers");
    const int n = b * b;
    const int nf = dict_id == AQMP_DICT_DCT_HAAR ? 2 : 1;
    const int M = nf * n;
    const int Mpad = (M + 127) / 128 * 128;
    const int Kpad = (n + kKBlock - 1) / kKBlock * kKBlock;
    const long long max_blocks = (long long)(kScratchBytes / ((size_t)Kpad * sizeof(__nv_bfloat16)));
    if (L > max_blocks)
        return set_error(AQMP_E_ARG, "aqmp_correlate_noalloc: more blocks than the static scratch holds");
    if (L == 0) return AQMP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // every call waits for its stream and reads a status word back, which a
    // stream capture cannot record: refuse before touching the stream
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess)
        return set_error(AQMP_E_CUDA, "aqmp_correlate_noalloc: cannot query the stream");
    if (cap != cudaStreamCaptureStatusNone)
        return set_error(AQMP_E_UNSUPPORTED, "aqmp_correlate_noalloc: the stream is being captured");

    std::lock_guard<std::mutex> lock(g_mu);
    Slot *slot;
    int rc = device_slot(&slot);
    if (rc != AQMP_OK) return rc;
    // Errors before the first enqueue return at once; errors after it wait
    // for the stream first, so that no work of this call still writes the
    // shared arrays when the next caller takes the lock.
    bool queued = false;
    auto fail_after = [&](int code, const char *msg) {
        if (queued) cudaStreamSynchronize(st);
        return set_error(code, msg);
    };
#define NA_CK(call)                                                                   \
    do {                                                                              \
        if ((call) != cudaSuccess) return fail_after(AQMP_E_CUDA, #call " failed");   \
    } while (0)

    // tensor maps first: they need only the arrays' addresses
    CUtensorMap ymap;
    if ((rc = bf16_tensor_map(&ymap, slot->scratch, (unsigned long long)L, Kpad, 64))) return rc;
    const bool rebuild = slot->table_b != b || slot->table_dict != dict_id;
    if (rebuild) {
        if ((rc = bf16_tensor_map(&slot->limb_map, slot->limbs, (unsigned long long)kLimbs * Mpad, Kpad, 128)))
            return rc;
        slot->table_b = 0;                      // the tables are stale until the rebuild completes
        slot->table_dict = -1;
        std::vector<double> basis;
        fp64_bases(b, basis);
        queued = true;
        NA_CK(cudaMemsetAsync(slot->limbs, 0, sizeof(g_limbs), st));
        NA_CK(cudaMemcpyAsync(slot->basis, basis.data(), sizeof(double) * basis.size(), cudaMemcpyHostToDevice, st));
        static_tables_kernel<<<(M + 7) / 8, 256, 0, st>>>(b, nf, dict_id == AQMP_DICT_HAAR ? 1 : 0,
                                                           (const double *)slot->basis, Mpad, Kpad,
                                                           (__nv_bfloat16 *)slot->limbs, (long long *)slot->sums);
        NA_CK(cudaGetLastError());
        NA_CK(cudaStreamSynchronize(st));       // the host basis buffer goes out of scope
        slot->table_b = b;
        slot->table_dict = dict_id;
    }
    queued = true;
    NA_CK(cudaMemsetAsync(slot->counters, 0, sizeof(Counters), st));
    // gather into the static scratch (every byte read below is rewritten)
    NA_CK(launch_gather_blocks(b, Kpad, blocks, L, (__nv_bfloat16 *)slot->scratch, nullptr, slot->sms, st));
    DictDev d{};
    d.b = b;
    d.n = n;
    d.M = M;
    d.Mpad = Mpad;
    d.Kpad = Kpad;
    d.nf = nf;
    d.limbs = (__nv_bfloat16 *)slot->limbs;
    d.Sh = (long long *)slot->sums;
    d.Sl = (long long *)slot->sums + kMaxAtoms;
    d.tmap_limbs = &slot->limb_map;
    CorrArgs ca{};
    ca.d = &d;
    ca.Y = (const __nv_bfloat16 *)slot->scratch;
    ca.count = nullptr;
    ca.fixed_count = L;
    ca.capacity = (unsigned)L;
    ca.c0 = (float2 *)corr;
    ca.ctr = (Counters *)slot->counters;
    ca.tmap_Y = &ymap;
    NA_CK(launch_corr_tc(ca, st));
    unsigned err = 0;
    NA_CK(cudaMemcpyAsync(&err, &((Counters *)slot->counters)->error, sizeof err, cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (err == kDevErrTimeout) return set_error(AQMP_E_TIMEOUT, "aqmp_correlate_noalloc: a bounded device wait gave up");
    if (err) return set_error(AQMP_E_CUDA, "aqmp_correlate_noalloc: device error");
#undef NA_CK
    return AQMP_OK;
}
