// codec.cu -- the codec stages around the encoder (Section 2.3, Appendix A):
// colour conversion entry points and the bitstream that the lossless stage
// (DEFLATE) compresses.  The bitstream layout is documented with
// aqmp_bitstream_write in aqmp.h; leaf positions are not stored, they follow
// from the depth-first order and the leaf sizes, as in the paper's decoder
// (Algorithm 3 places each block by the quadtree traversal order).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <vector>

#include "../../include/aqmp.h"
#include "code.h"
#include "common.cuh"
#include "kernels.h"

using namespace aqmp;

namespace {

constexpr uint8_t kMagic[4] = {'A', 'Q', 'M', 'P'};
constexpr int kVersion = 1;
constexpr size_t kHeaderBytes = 16;
constexpr size_t kPlaneBytes = 16;

int log2i(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

size_t varint_len(uint32_t v) {
    size_t n = 1;
    while (v >= 0x80u) { v >>= 7; ++n; }
    return n;
}

struct Writer {
    uint8_t *p, *end;
    bool ok = true;
    void bytes(const void *src, size_t n) {
        if ((size_t)(end - p) < n) { ok = false; return; }
        std::memcpy(p, src, n);
        p += n;
    }
    void u8(uint8_t v) { bytes(&v, 1); }
    void u16(uint16_t v) { uint8_t b[2] = {(uint8_t)v, (uint8_t)(v >> 8)}; bytes(b, 2); }
    void u32(uint32_t v) {
        uint8_t b[4] = {(uint8_t)v, (uint8_t)(v >> 8), (uint8_t)(v >> 16), (uint8_t)(v >> 24)};
        bytes(b, 4);
    }
    void f32(float f) { uint32_t v; std::memcpy(&v, &f, 4); u32(v); }
    void varint(uint32_t v) {
        while (v >= 0x80u) { u8((uint8_t)(v | 0x80u)); v >>= 7; }
        u8((uint8_t)v);
    }
};

struct Reader {
    const uint8_t *p, *end;
    bool ok = true;
    bool take(void *dst, size_t n) {
        if (!ok || (size_t)(end - p) < n) { ok = false; return false; }
        std::memcpy(dst, p, n);
        p += n;
        return true;
    }
    uint8_t u8() { uint8_t v = 0; take(&v, 1); return v; }
    uint16_t u16() { uint8_t b[2] = {0, 0}; take(b, 2); return (uint16_t)(b[0] | (b[1] << 8)); }
    uint32_t u32() {
        uint8_t b[4] = {0, 0, 0, 0};
        take(b, 4);
        return (uint32_t)b[0] | ((uint32_t)b[1] << 8) | ((uint32_t)b[2] << 16) | ((uint32_t)b[3] << 24);
    }
    float f32() { uint32_t v = u32(); float f; std::memcpy(&f, &v, 4); return f; }
    uint32_t varint() {
        uint32_t v = 0;
        for (int shift = 0; shift < 35; shift += 7) {
            const uint8_t b = u8();
            if (!ok) return 0;
            v |= (uint32_t)(b & 0x7fu) << shift;
            if (!(b & 0x80u)) return v;
        }
        ok = false;
        return 0;
    }
};

struct PlaneHead { uint32_t h, w, n_leaves, n_atoms; };

// Host copies of a code's arrays (canonical order) and the per-plane ranges.
int host_arrays(const aqmp_code *code, std::vector<LeafRec> &L, std::vector<AtomRec> &A) {
    L.resize(code->n_leaves);
    A.resize(code->n_atoms);
    if (code->n_leaves &&
        cudaMemcpy(L.data(), code->leaves, sizeof(LeafRec) * L.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return set_error(AQMP_E_CUDA, "device-to-host copy of the leaves failed");
    if (code->n_atoms &&
        cudaMemcpy(A.data(), code->atoms, sizeof(AtomRec) * A.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return set_error(AQMP_E_CUDA, "device-to-host copy of the atoms failed");
    return AQMP_OK;
}

// Size of the bitstream from the per-leaf step counts.
uint64_t stream_bytes(const aqmp_code *code, const std::vector<LeafRec> &L) {
    uint64_t n = kHeaderBytes + kPlaneBytes * code->shapes.size();
    for (const LeafRec &r : L) n += 1 + varint_len(r.n_atoms) + 6ull * r.n_atoms;
    return n;
}

// Parse into host arrays; positions recovered by walking each root's
// quadtree depth-first (TL, TR, BL, BR) against the listed leaf sizes.
int parse(const uint8_t *buf, uint64_t len, aqmp_bitstream_info &info, std::vector<PlaneHead> &heads,
          std::vector<LeafRec> *L, std::vector<AtomRec> *A) {
    if (!buf) return set_error(AQMP_E_ARG, "malformed bitstream: NULL buffer");
    Reader r{buf, buf + len};
    uint8_t magic[4] = {0, 0, 0, 0};
    r.take(magic, 4);
    if (!r.ok || std::memcmp(magic, kMagic, 4) != 0) return set_error(AQMP_E_ARG, "malformed bitstream: bad magic");
    info = aqmp_bitstream_info{};
    info.version = r.u8();
    info.color = r.u8();
    info.dict_id = r.u8();
    r.u8();
    info.min_block = r.u16();
    info.max_block = r.u16();
    const uint32_t np = r.u32();
    if (!r.ok || info.version != kVersion) return set_error(AQMP_E_ARG, "malformed bitstream: bad header");
    if (info.color < 0 || info.color > 2 || info.dict_id < 0 || info.dict_id > 2)
        return set_error(AQMP_E_ARG, "malformed bitstream: bad colour or dictionary");
    const int mb = info.max_block, nb = info.min_block;
    if (nb < 1 || mb < nb || mb > kMaxSide || (mb & (mb - 1)) || (nb & (nb - 1)))
        return set_error(AQMP_E_ARG, "malformed bitstream: bad block sizes");
    if ((uint64_t)np * kPlaneBytes > len) return set_error(AQMP_E_ARG, "malformed bitstream: truncated");
    info.n_planes = (int)np;
    heads.resize(np);
    for (auto &h : heads) {
        h.h = r.u32();
        h.w = r.u32();
        h.n_leaves = r.u32();
        h.n_atoms = r.u32();
        if (!r.ok || h.h == 0 || h.w == 0 || h.h % mb || h.w % mb)
            return set_error(AQMP_E_ARG, "malformed bitstream: bad plane shape");
        info.n_leaves += h.n_leaves;
        info.n_atoms += h.n_atoms;
    }
    if (!L) return AQMP_OK;
    if (info.n_leaves > len || info.n_atoms > len) return set_error(AQMP_E_ARG, "malformed bitstream: truncated");
    L->clear();
    A->clear();
    L->reserve(info.n_leaves);
    A->reserve(info.n_atoms);
    struct Node { uint32_t y, x, b; };
    std::vector<Node> stack;
    const int maxlev = log2i(mb / nb);
    for (uint32_t p = 0; p < np; ++p) {
        const PlaneHead &h = heads[p];
        const uint8_t *levels = r.p;
        if ((uint64_t)(r.end - r.p) < h.n_leaves) return set_error(AQMP_E_ARG, "malformed bitstream: truncated");
        r.p += h.n_leaves;
        const size_t first = L->size();
        uint32_t next = 0;
        for (uint32_t ry = 0; ry < h.h / mb; ++ry) {
            for (uint32_t rx = 0; rx < h.w / mb; ++rx) {
                stack.assign(1, Node{ry * (uint32_t)mb, rx * (uint32_t)mb, (uint32_t)mb});
                while (!stack.empty()) {
                    Node n = stack.back();
                    stack.pop_back();
                    if (next >= h.n_leaves) return set_error(AQMP_E_ARG, "malformed bitstream: too few leaves");
                    const int lev = levels[next];
                    if (lev > maxlev) return set_error(AQMP_E_ARG, "malformed bitstream: bad leaf size");
                    const uint32_t b = (uint32_t)mb >> lev;
                    if (b > n.b) return set_error(AQMP_E_ARG, "malformed bitstream: leaf larger than its node");
                    if (b < n.b) {
                        const uint32_t c = n.b / 2;
                        stack.push_back(Node{n.y + c, n.x + c, c});     // BR
                        stack.push_back(Node{n.y + c, n.x, c});         // BL
                        stack.push_back(Node{n.y, n.x + c, c});         // TR
                        stack.push_back(Node{n.y, n.x, c});             // TL, visited next
                        continue;
                    }
                    LeafRec rec{};
                    rec.plane = p;
                    rec.y = n.y;
                    rec.x = n.x;
                    rec.b = (uint16_t)b;
                    L->push_back(rec);
                    ++next;
                }
            }
        }
        if (next != h.n_leaves) return set_error(AQMP_E_ARG, "malformed bitstream: leaves do not tile the plane");
        uint64_t atoms = 0;
        for (size_t i = first; i < L->size(); ++i) {
            const uint32_t t = r.varint();
            LeafRec &rec = (*L)[i];
            const int n = (int)rec.b * rec.b;
            const int k_max = (info.dict_id == AQMP_DICT_DCT_HAAR ? 2 : 1) * n;
            if (!r.ok || t > 0xffffu || (int)t > k_max) return set_error(AQMP_E_ARG, "malformed bitstream: bad step count");
            rec.n_atoms = (uint16_t)t;
            rec.atom_off = (uint32_t)(A->size() + atoms);
            atoms += t;
        }
        if (atoms != h.n_atoms) return set_error(AQMP_E_ARG, "malformed bitstream: atom count mismatch");
        const size_t a0 = A->size();
        A->resize(a0 + atoms);
        for (uint64_t i = 0; i < atoms; ++i) (*A)[a0 + i].j = r.u16();
        for (uint64_t i = 0; i < atoms; ++i) (*A)[a0 + i].alpha = r.f32();
        if (!r.ok) return set_error(AQMP_E_ARG, "malformed bitstream: truncated");
        for (size_t i = first; i < L->size(); ++i) {
            const LeafRec &rec = (*L)[i];
            const uint32_t m = (uint32_t)(info.dict_id == AQMP_DICT_DCT_HAAR ? 2 : 1) * rec.b * rec.b;
            for (uint32_t t = 0; t < rec.n_atoms; ++t)
                if ((*A)[rec.atom_off + t].j >= m) return set_error(AQMP_E_ARG, "malformed bitstream: atom index");
        }
    }
    if (r.p != r.end) return set_error(AQMP_E_ARG, "malformed bitstream: trailing bytes");
    return AQMP_OK;
}

}  // namespace

extern "C" {

int aqmp_image_to_planes(const uint8_t *img, int h, int w, int channels, int64_t pitch, int color, uint8_t *planes,
                         int64_t plane_pitch, void *stream) {
    if (!img || !planes || h <= 0 || w <= 0 || channels <= 0 || pitch < (int64_t)w * channels || plane_pitch < w)
        return set_error(AQMP_E_ARG, "aqmp_image_to_planes: bad pointer or shape");
    if (color < 0 || color > 2 || (color == AQMP_COLOR_YCBCR && channels != 3))
        return set_error(AQMP_E_ARG, "aqmp_image_to_planes: YCbCr needs 3 channels");
    int sms = 0;
    int rc = device_sm_count(&sms);
    if (rc) return rc;
    ColorArgs a{};
    a.img = img;
    a.pitch = pitch;
    a.planes_u8 = planes;
    a.plane_pitch = plane_pitch;
    a.h = h;
    a.w = w;
    a.channels = channels;
    a.color = color;
    cudaError_t e = launch_color(a, true, sms, (cudaStream_t)stream);
    return e == cudaSuccess ? AQMP_OK : set_error(AQMP_E_CUDA, cudaGetErrorString(e));
}

int aqmp_planes_to_image(const float *planes, int h, int w, int channels, int64_t plane_pitch, int color, uint8_t *img,
                         int64_t pitch, void *stream) {
    if (!img || !planes || h <= 0 || w <= 0 || channels <= 0 || pitch < (int64_t)w * channels || plane_pitch < w)
        return set_error(AQMP_E_ARG, "aqmp_planes_to_image: bad pointer or shape");
    if (color < 0 || color > 2 || (color == AQMP_COLOR_YCBCR && channels != 3))
        return set_error(AQMP_E_ARG, "aqmp_planes_to_image: YCbCr needs 3 channels");
    int sms = 0;
    int rc = device_sm_count(&sms);
    if (rc) return rc;
    ColorArgs a{};
    a.img_out = img;
    a.pitch = pitch;
    a.planes_f32 = planes;
    a.plane_pitch = plane_pitch;
    a.h = h;
    a.w = w;
    a.channels = channels;
    a.color = color;
    cudaError_t e = launch_color(a, false, sms, (cudaStream_t)stream);
    return e == cudaSuccess ? AQMP_OK : set_error(AQMP_E_CUDA, cudaGetErrorString(e));
}

int aqmp_bitstream_size(const aqmp_code *code, uint64_t *bytes) {
    if (!code || !bytes) return set_error(AQMP_E_ARG, "NULL argument");
    std::vector<LeafRec> L;
    std::vector<AtomRec> A;
    int rc = host_arrays(code, L, A);
    if (rc) return rc;
    *bytes = stream_bytes(code, L);
    return AQMP_OK;
}

int aqmp_bitstream_write(const aqmp_code *code, int color, uint8_t *buf, uint64_t cap, uint64_t *len) {
    if (!code || !buf || !len) return set_error(AQMP_E_ARG, "NULL argument");
    if (color < 0 || color > 2) return set_error(AQMP_E_ARG, "bad colour mode");
    std::vector<LeafRec> L;
    std::vector<AtomRec> A;
    int rc = host_arrays(code, L, A);
    if (rc) return rc;
    const uint64_t need = stream_bytes(code, L);
    if (cap < need) return set_error(AQMP_E_ARG, "bitstream buffer too small");
    const size_t np = code->shapes.size();
    std::vector<size_t> lbeg(np + 1, 0);
    std::vector<PlaneHead> heads(np);
    for (size_t p = 0; p < np; ++p) {
        heads[p].h = (uint32_t)code->shapes[p].first;
        heads[p].w = (uint32_t)code->shapes[p].second;
    }
    for (const LeafRec &r : L) {
        if (r.plane >= np) return set_error(AQMP_E_ARG, "leaf of an unknown plane");
        heads[r.plane].n_leaves += 1;
        heads[r.plane].n_atoms += r.n_atoms;
    }
    Writer wr{buf, buf + cap};
    wr.bytes(kMagic, 4);
    wr.u8((uint8_t)kVersion);
    wr.u8((uint8_t)color);
    wr.u8((uint8_t)code->dict_id);
    wr.u8(0);
    wr.u16((uint16_t)code->min_block);
    wr.u16((uint16_t)code->max_block);
    wr.u32((uint32_t)np);
    for (const PlaneHead &h : heads) {
        wr.u32(h.h);
        wr.u32(h.w);
        wr.u32(h.n_leaves);
        wr.u32(h.n_atoms);
    }
    // leaves are plane-major in canonical order, so each plane is one range
    size_t i = 0;
    for (size_t p = 0; p < np; ++p) {
        const size_t b0 = i;
        while (i < L.size() && L[i].plane == p) ++i;
        const int top = log2i(code->max_block);
        for (size_t k = b0; k < i; ++k) wr.u8((uint8_t)(top - log2i(L[k].b)));
        for (size_t k = b0; k < i; ++k) wr.varint(L[k].n_atoms);
        for (size_t k = b0; k < i; ++k)
            for (uint32_t t = 0; t < L[k].n_atoms; ++t) wr.u16((uint16_t)A[L[k].atom_off + t].j);
        for (size_t k = b0; k < i; ++k)
            for (uint32_t t = 0; t < L[k].n_atoms; ++t) wr.f32(A[L[k].atom_off + t].alpha);
    }
    if (i != L.size()) return set_error(AQMP_E_ARG, "leaves are not in plane order");
    if (!wr.ok) return set_error(AQMP_E_ARG, "bitstream buffer too small");
    *len = (uint64_t)(wr.p - buf);
    return AQMP_OK;
}

int aqmp_bitstream_parse(const uint8_t *buf, uint64_t len, aqmp_bitstream_info *info, int *shapes,
                         aqmp_leaf *leaves, aqmp_atom *atoms) {
    if (!info) return set_error(AQMP_E_ARG, "NULL argument");
    std::vector<PlaneHead> heads;
    std::vector<LeafRec> L;
    std::vector<AtomRec> A;
    const bool want = leaves || atoms;
    int rc = parse(buf, len, *info, heads, want ? &L : nullptr, want ? &A : nullptr);
    if (rc) return rc;
    if (shapes)
        for (size_t p = 0; p < heads.size(); ++p) {
            shapes[2 * p] = (int)heads[p].h;
            shapes[2 * p + 1] = (int)heads[p].w;
        }
    if (leaves && !L.empty()) std::memcpy(leaves, L.data(), sizeof(LeafRec) * L.size());
    if (atoms && !A.empty()) std::memcpy(atoms, A.data(), sizeof(AtomRec) * A.size());
    return AQMP_OK;
}

int aqmp_code_from_bitstream(const uint8_t *buf, uint64_t len, aqmp_code **out) {
    if (!out) return set_error(AQMP_E_ARG, "NULL argument");
    *out = nullptr;
    aqmp_bitstream_info info{};
    std::vector<PlaneHead> heads;
    std::vector<LeafRec> L;
    std::vector<AtomRec> A;
    int rc = parse(buf, len, info, heads, &L, &A);
    if (rc) return rc;
    auto code = std::make_unique<aqmp_code>();
    if (cudaGetDevice(&code->device) != cudaSuccess) return set_error(AQMP_E_CUDA, "no CUDA device");
    code->dict_id = info.dict_id;
    code->min_block = info.min_block;
    code->max_block = info.max_block;
    for (const PlaneHead &h : heads) code->shapes.emplace_back((int)h.h, (int)h.w);
    code->n_leaves = L.size();
    code->n_atoms = A.size();
    const size_t nl = std::max<size_t>(1, L.size()), na = std::max<size_t>(1, A.size());
    if (cudaMalloc((void **)&code->leaves, sizeof(LeafRec) * nl) != cudaSuccess ||
        cudaMalloc((void **)&code->atoms, sizeof(AtomRec) * na) != cudaSuccess ||
        cudaMalloc((void **)&code->alpha_lo, sizeof(float) * na) != cudaSuccess)
        return set_error(AQMP_E_OOM, "cudaMalloc for the code arrays failed");
    if ((!L.empty() && cudaMemcpy(code->leaves, L.data(), sizeof(LeafRec) * L.size(), cudaMemcpyHostToDevice)) ||
        (!A.empty() && cudaMemcpy(code->atoms, A.data(), sizeof(AtomRec) * A.size(), cudaMemcpyHostToDevice)) ||
        cudaMemset(code->alpha_lo, 0, sizeof(float) * na) != cudaSuccess)
        return set_error(AQMP_E_CUDA, "upload of the code arrays failed");
    aqmp_stats &s = code->stats;
    s.n_leaves = L.size();
    s.n_atoms = A.size();
    *out = code.release();
    return AQMP_OK;
}

}  // extern "C"
