// kernels.h -- argument blocks and launchers of the AQMP device kernels.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <vector>

#include "common.cuh"

namespace aqmp {

// Pursuit of one level (mp.cu).
struct MPArgs {
    LevelArgs lv;
    const float2 *c0;            // [capacity][M] initial correlations (hi, lo)
    const uint32_t *e0;          // [capacity] sum of squared pixels of each block
    const PlaneDesc *planes;
    const float2 *W;             // W = C H^T, b x b row-major, (hi, lo) pairs
    const float2 *WT;            // its transpose
    LeafRec *leaves;
    unsigned long long leaf_cap;
    AtomRec *atoms;
    float *alpha_lo;
    uint32_t *atom_leaf;         // emission slot of the leaf owning each atom
    unsigned long long atom_cap;
    CellMap cells;               // emitted leaves are marked here
    Counters *ctr;
    // OMP at sides 32 and 64: one packed Cholesky factor of up to k(k+1)/2
    // doubles per CTA, omp_slots of them (omp_L_doubles in all)
    double *omp_L;
    int omp_slots;
    unsigned long long omp_L_doubles;
    // the BF16 form with rescore (side 64; ebound NULL: off): the BF16
    // correlation's per-atom bounds, the leaves' mean-centred pixels and their
    // centres, the exact form's fixed-point rows and row sums, and the queue
    // of leaves handed to the exact path
    const float *ebound;
    const __nv_bfloat16 *Yc;
    int Kpad;
    const uint8_t *mu;
    const int2 *Bs;
    const long long *Rs;
    QueueEntry *fb_queue;
    unsigned *fb_count;
    unsigned fb_capacity;
    unsigned *work;              // leaf counter (NULL: ctr->work_next[level])
    int fam0;                    // family of a single-family dictionary
};
// variant 0: the default launch shape; 1: the alternate one (other threads
// per leaf at sides 16 and 32, two resident CTAs per SM at side 64; two
// families only, the same as 0 elsewhere).  Both give the same result bit
// for bit.
cudaError_t launch_mp(const MPArgs &a, int nf, bool double_float, int variant, int num_sms, cudaStream_t st);
bool mp_has_variant(int b, int nf);
// Side 128 (mp_cluster.cu): one leaf per cluster of 2 nf CTAs, same
// arguments and outputs as launch_mp.
cudaError_t launch_mp_cluster(const MPArgs &a, int nf, bool double_float, int num_sms, cudaStream_t st);

// Orthogonal Matching Pursuit of one level: sides 4, 8, 16 with a warp per
// leaf (omp.cu), sides 32 and 64 with a CTA per leaf and the Cholesky factor
// in the omp_L slots (omp_cta.cu); budget k <= omp_max_budget(b) (0: side not
// served); same arguments and outputs as the MP kernel (the coefficients
// emitted are the final least-squares values).
int omp_max_budget(int b);
unsigned long long omp_cta_workspace_doubles(int k, int slots);
cudaError_t launch_omp(const MPArgs &a, int nf, int num_sms, cudaStream_t st);
int omp_cta_max_budget();
cudaError_t launch_omp_cta(const MPArgs &a, int nf, cudaStream_t st);

// Block gather (gather.cu): queue entries -> centred BF16 leaf vectors
// (column-major unravel, zero padded to Kpad) and sums of squares.
struct GatherArgs {
    int b, n, Kpad;
    const QueueEntry *queue;
    const unsigned *count;
    unsigned capacity;
    const PlaneDesc *planes;
    __nv_bfloat16 *Y;            // [capacity][Kpad]
    uint32_t *e0;                // [capacity]
    uint8_t *Y8;                 // FP8 form: e4m3(y~ s_l) [capacity][kpad_fp8(n)], or NULL
    float *inv_sl;               // FP8 form: 1 / s_l per leaf
    uint8_t *mu;                 // BF16 form with rescore: centre on the block's integer
                                 // mean, written here per leaf (NULL: centre 128)
};
cudaError_t launch_gather(const GatherArgs &a, int num_sms, cudaStream_t st);

// Same, for L contiguous row-major b x b blocks (aqmp_correlate).
cudaError_t launch_gather_blocks(int b, int Kpad, const uint8_t *blocks, long long L,
                                 __nv_bfloat16 *Y, uint32_t *e0, int num_sms, cudaStream_t st,
                                 uint8_t *mu = nullptr);
cudaError_t launch_gather_blocks_fp8(int b, const uint8_t *blocks, long long L, uint8_t *Y8, float *inv_sl,
                                     int num_sms, cudaStream_t st);

// Fixed-point dictionary tables of one side (tables.cu).
struct DictDev {
    int b, n, M, Mpad, Kpad, nf;
    int fam0;                    // family of a single-family dictionary (0 = DCT, 1 = Haar)
    // separable fixed-point dictionary (sep.cuh), both families always:
    int2 *Bs;                    // [2][b][b] Bf[F][p][i] as 24-bit limbs (lo, hi)
    int2 *BsT;                   // [2][b][b] its transpose, BsT[F][m][q] = Bf[F][q][m]
    long long *Rs;               // [2][b] row sums R[F][p] = sum_i Bf[F][p][i]
    __nv_bfloat16 *sepd;         // side 64: Bf digits for the tensor cores (corr_sep_tc.cu)
    void *tmap_sepd;             // its CUtensorMap (host copy)
    // side 64, the BF16 form with rescore: [bf16(B_F); bf16(B_F - bf16(B_F))]
    // for F = 0, 1, then [|B_0|; |B_1|] rounded up, each 128 rows x b BF16
    __nv_bfloat16 *sepbf;
    void *tmap_sepbf;            // its CUtensorMap (host copy), boxes of 128 rows
    float2 *Rbf;                 // [2][b] row sums sum_i B[F][p][i] as (hi, lo)
    __nv_bfloat16 *limbs;        // [kLimbs][Mpad][Kpad] balanced base-64 digits
    int32_t *Dh, *Dl;            // [M][n]: D_fix = Dh 2^24 + Dl, Dl in [-2^23, 2^23)
    long long *Sh, *Sl;          // per atom: sum_v D_fix = Sh 2^24 + Sl (canonical)
    float2 *W, *WT;              // b x b (hi, lo)
    float *basis;                // [2][b][b] FP32 1-D bases (DCT, Haar) for decoding
    void *tmap_limbs;            // CUtensorMap for the tensor-core kernel (host copy)
    __nv_bfloat16 *Dbf;          // [Mpad][Kpad] bf16(D) (reduced-precision form; built on demand)
    float *Sbf;                  // [M] row sums of bf16(D)
    void *tmap_bf16;             // CUtensorMap of Dbf (host copy)
    // FP8 form (built on demand): e4m3(D[j][v] s_j) with a power-of-two scale
    // per atom, its inverse and the row sums of the dequantised entries
    uint8_t *D8;                 // [Mpad][K8] e4m3 bytes, K8 = kpad_fp8(n)
    float *inv_s8;               // [M] 1 / s_j
    float *S8;                   // [M] sum_v e4m3(D[j][v] s_j) / s_j
    void *tmap_fp8;              // CUtensorMap of D8 (host copy)
};

// K padding of the FP8 form: one 128-byte swizzle row holds 128 elements.
__host__ __device__ inline int kpad_fp8(int n) { return n < 128 ? 128 : (n + 127) / 128 * 128; }

// Initial correlation (corr_simt.cu / corr_tc.cu): c0[l][j] for l < *count.
struct CorrArgs {
    const DictDev *d;            // host pointer to the table descriptor
    const __nv_bfloat16 *Y;      // [capacity][Kpad]
    const unsigned *count;       // device count (NULL: use `fixed_count`)
    long long fixed_count;
    unsigned capacity;
    float2 *c0;                  // [capacity][M]
    Counters *ctr;               // may be NULL
    const void *tmap_Y;          // CUtensorMap of Y (tensor-core kernel only)
    const void *tmap_Ysep;       // Y as [capacity b][b] rows (separable tensor-core kernels)
    // BF16 form with rescore: the per-leaf centres and the per-atom bounds
    const uint8_t *mu;           // [capacity] integer mean each leaf's Y is centred on
    float *ebound;               // [capacity][M] bound on |c0 - the exact form's c0|
    // separable exact kernels: the families (bit F: 0 DCT-II, 1 Haar) this
    // launch computes, 0 = all of the dictionary's; the others' outputs are
    // left as they are (the layout is always the dictionary's [capacity][M])
    int fmask;
};
cudaError_t launch_corr_simt(const CorrArgs &a, cudaStream_t st);
// Exact correlation with the separable fixed-point dictionary (corr_sep.cu):
// B Y B^T per family in integers, T 2^-96 rounded once into a double-float.
cudaError_t launch_corr_sep_simt(const CorrArgs &a, cudaStream_t st);
// The same on the tensor cores (corr_sep_tc.cu), bit for bit, at the sides
// where corr_sep_tc_available() says a kernel exists.
cudaError_t launch_corr_sep_tc(const CorrArgs &a, cudaStream_t st);
bool corr_sep_tc_available(int b, int nf);
// BF16 form with rescore (corr_sepbf_tc.cu): c0 from split BF16 products of
// the separable form, Y centred on a.mu, and the per-atom bound a.ebound.
bool corr_sepbf_available(int b);
cudaError_t launch_corr_sepbf(const CorrArgs &a, cudaStream_t st);
cudaError_t launch_corr_tc(const CorrArgs &a, cudaStream_t st);
// Reduced-precision form: one BF16 pass of bf16(D), FP32 accumulation (c0 low words 0).
cudaError_t launch_corr_tc_bf16(const CorrArgs &a, cudaStream_t st);
// FP8 form: one E4M3 pass (kind::f8f6f4) of the per-atom scaled e4m3(D)
// against the per-leaf scaled e4m3 pixels, FP32 accumulation, rescaled.
cudaError_t launch_corr_tc_fp8(const CorrArgs &a, const float *inv_sl, cudaStream_t st);
bool corr_tc_available();
cudaError_t launch_wait_selftest(Counters *ctr, unsigned long long limit_ns, cudaStream_t st);

// Decoder (decode.cu): one plane's leaves -> float image.
struct DecodeArgs {
    const LeafRec *leaves;
    unsigned long long n_leaves;
    const AtomRec *atoms;
    uint32_t plane;
    float *out;
    long long out_pitch;
    const float *basis[8];       // per level log2(b): [2][b][b] FP32 bases
    int nf;                      // 2: DCT+Haar, 1: single family
    int single_family;           // 0: DCT, 1: Haar (when nf == 1)
};
cudaError_t launch_decode(const DecodeArgs &a, int num_sms, cudaStream_t st);
// The same with caller coefficients alpha[atom] in place of the code's.
cudaError_t launch_decode_alpha(const DecodeArgs &a, const float *alpha, int num_sms, cudaStream_t st);

// Refinement on a fixed support (diff.cu).
cudaError_t upload_gauss11(cudaStream_t st);
cudaError_t launch_synth_forward(const LeafRec *leaves, unsigned long long n_leaves, const AtomRec *atoms,
                                 const float *alpha, uint32_t plane, float *out, long long pitch,
                                 const DecodeArgs &bases, int num_sms, cudaStream_t st);
cudaError_t launch_synth_backward(const LeafRec *leaves, unsigned long long n_leaves, const AtomRec *atoms,
                                  uint32_t plane, const float *grad, long long pitch, float *grad_alpha,
                                  const DecodeArgs &bases, int max_side, int num_sms, cudaStream_t st);
cudaError_t launch_ssim(const float *x, const float *y, int h, int w, long long pitch, double *H, double *P,
                        double *V, double *sum, float *grad, double gscale, int num_sms, cudaStream_t st);

// Level-0 queue from the plane descriptors (gather.cu).
cudaError_t launch_seed_roots(const PlaneDesc *planes, int n_planes, int max_block,
                              unsigned total_roots, QueueEntry *queue, unsigned *count,
                              cudaStream_t st);

// Canonical (depth-first) order of the emitted leaves (order.cu), three
// launches over the cell map the pursuit kernels filled: phase 0 ranks the
// leaves (perm[rank] = slot), phase 1 writes the ordered records and each
// slot's new atom offset, phase 2 moves every atom.  Phases 0 and 1 are
// single-pass scans with decoupled look-back over tiles claimed in launch
// order; `status` (order_status_words(n_cells, leaf_cap) 64-bit words) must
// be zero before phase 0.
struct OrderOut {                      // read from device memory, so that a captured
    LeafRec *leaves;                   // graph serves calls with different outputs
    AtomRec *atoms;
    float *lo;
};
struct OrderArgs {
    CellMap cells;
    const LeafRec *leaves_in;
    const AtomRec *atoms_in;
    const float *lo_in;
    const uint32_t *atom_leaf;         // slot of each emitted atom's leaf
    const unsigned long long *n_leaves, *n_atoms;
    unsigned long long leaf_cap, atom_cap;
    uint32_t *perm;                    // leaf_cap words
    uint32_t *new_off;                 // leaf_cap words: new atom offset by slot
    unsigned long long *status;
    const OrderOut *out;               // device: the call's output arrays
    Counters *ctr;
    unsigned long long limit_ns;       // bound on every look-back wait
};
unsigned long long order_status_words(unsigned long long n_cells, unsigned long long leaf_cap);
cudaError_t launch_order_phase(const OrderArgs &a, int phase, int num_sms, cudaStream_t st);

// Colour conversion of the codec (color.cu): an interleaved h x w x C byte
// image <-> C planes (plane c at c h plane_pitch); color 2 = YCbCr <-> RGB
// (C = 3), otherwise the channels are copied.  Planes going out are bytes,
// planes coming back are the decoder's floats.
struct ColorArgs {
    const uint8_t *img;
    uint8_t *img_out;
    long long pitch;
    uint8_t *planes_u8;
    const float *planes_f32;
    long long plane_pitch;
    int h, w, channels, color;
};
cudaError_t launch_color(const ColorArgs &a, bool to_planes, int num_sms, cudaStream_t st);

// Table construction on the device (tables.cu) from the FP64 1-D bases
// basis_dev = [2][b][b] (DCT, Haar); fam0 selects the family of a
// single-family dictionary (0 = DCT, 1 = Haar).
cudaError_t build_fixed_tables_fam(DictDev &d, const double *basis_dev, int fam0, cudaStream_t st);
// bf16(D) and its row sums for the reduced-precision form.
cudaError_t build_bf16_tables(DictDev &d, const double *basis_dev, int fam0, cudaStream_t st);
// e4m3(D s_j), 1 / s_j and the dequantised row sums for the FP8 form.
cudaError_t build_fp8_tables(DictDev &d, const double *basis_dev, int fam0, cudaStream_t st);
// FP32 copy of the FP64 bases (decoder tables).
cudaError_t launch_basis_to_float(const double *basis_dev, float *out, int count, cudaStream_t st);

// Host helpers defined in host.cu for the library's other entry points.
int set_error(int code, const char *msg);
void fp64_bases(int b, std::vector<double> &basis);
int bf16_tensor_map(void *map, const void *base, unsigned long long rows, unsigned long long cols,
                    unsigned box_rows);
int device_sm_count(int *sms);

}  // namespace aqmp
