// Mixed-precision form: double-float collocation, Ozaki-sliced (5 x 7-bit) bf16 tcgen05
// contractions with exact fp32 accumulator levels in tensor memory, float64 weights,
// functional and accumulation.
#pragma once

#include <cstdint>
#include <vector>

#include "internal.h"

namespace gbxc {

size_t fp64_row_bytes();
void append_fp64_vtasks(int j, int n, int64_t s0, int64_t s1, std::vector<int> &tasks);

// Per-context state of the mixed form: tensor-map encoder, the sliced P^j blocks of the
// current chunk and a device error word for bounded waits.
struct MixedCtx {
    void *encode_fn = nullptr;         // cuTensorMapEncodeTiled from the driver
    uint16_t *pslices = nullptr;       // 5 planes x rows x 32 bf16
    size_t pslice_rows = 0;            // capacity of pslices in elements
    float *pdf = nullptr;              // the P region (pdf_region_bytes): pairs, slices, exponents
    size_t pdf_cap = 0;
    // spin-unrestricted form: P_b's planes, the second X/Z slab and its Z exponents
    float *pdf2 = nullptr;
    size_t pdf2_cap = 0;
    float2 *x2 = nullptr;
    size_t x2_cap = 0;
    int *zexp2 = nullptr;
    size_t zexp2_cap = 0;
    // meta-GGA: slices of d_k Phi, the Y^k / W^k planes and their exponents, for chunks of
    // up to mgga_rows slab rows
    uint16_t *ax_g = nullptr;          // 3 x 5 planes x rows x 128 bf16
    float2 *y_g = nullptr;             // 3 planes x rows x 128
    int *pexp_g = nullptr;             // 3 x 4 rows point exponents
    int *wexp_g = nullptr, *gexp_g = nullptr;   // 3 x rows each
    size_t ax_g_cap = 0, y_g_cap = 0, pexp_g_cap = 0, wexp_g_cap = 0, gexp_g_cap = 0;
    int64_t mgga_rows = 0;
    int num_sms = 0;                   // persistent-GEMM grid size
    int keep_z = 0;                    // spin-restricted chunks also leave Z in the X plane
    int *d_err = nullptr;              // [0] error word of the bounded waits, [1] GEMM task counter
};
// A shell with every constant split into a double-float pair (hi + lo).
struct DfShell {
    float ch[3], cl[3];                               // centre
    float ah[GBXC_MAX_PRIM], al[GBXC_MAX_PRIM];       // exponents alpha
    float dh[GBXC_MAX_PRIM], dl[GBXC_MAX_PRIM];       // coefficients d
    float gh[GBXC_MAX_PRIM], gl[GBXC_MAX_PRIM];       // -2 alpha d (gradient coefficients)
    int L, nprim, fofs, pure;
};
// Per-molecule resident state of the mixed form.
struct MixedResident {
    DfShell *d_shells = nullptr;
    bool has_pure = false;   // any spherical shell: the collocation with the pure-shell path
};
cudaError_t build_mixed_resident(const std::vector<DevShell> &shells, MixedResident &r);
// Per-schedule state of the mixed form: for every chunk the batch range and the row
// offsets of each batch's sliced P^j block.
struct MixedSchedule {
    struct Chunk {
        int j0, j1;                    // batches touched by the chunk (inclusive)
        int64_t prow0;                 // offset of the chunk's entries in d_pofs
        int64_t prows;                 // rows of the sliced P^j blocks of the chunk
        int max_np;
        int64_t xtask0, nxtask;        // X-contraction tasks (tile, N chunk) of the chunk
        int64_t ptask0, nptask;        // P^j slicing tasks (batch, group of 8 rows) of the chunk
        int max_group = 8;             // tiles of the chunk's largest V task (z_slice's shared memory)
    };
    std::vector<Chunk> chunks;
    int *d_xtasks = nullptr;           // (tile, N chunk) pairs of every chunk
    int *d_ptasks = nullptr;           // (batch within the chunk, first row) pairs of every chunk
    int64_t *d_pofs = nullptr;         // per (chunk, batch): first P-slice row
    int64_t max_prows = 0;
    int bn = 128;                      // N tile of the tcgen05 GEMMs: 128 or 64 functions
};

size_t mixed_row_bytes();
// The P region of the tensor-core form, prepared once per integration from P (nbf x nbf):
// the (hi, lo) double-float pair of every element (8 nbf^2 bytes), then the 5 bf16 slices of
// every element with one exponent per row, as 16 bytes per element (slices 0-4, then three
// zero halves; element (mu, nu) at 8 (mu nbf + nu) halves, 16-byte aligned), then the row
// exponents (nbf ints).
__host__ __device__ inline size_t pdf_slices_offset(int nbf) { return ((size_t)8 * nbf * nbf + 15) & ~(size_t)15; }
__host__ __device__ inline size_t pdf_exps_offset(int nbf) { return pdf_slices_offset(nbf) + (size_t)16 * nbf * nbf; }
__host__ __device__ inline size_t pdf_region_bytes(int nbf) { return pdf_exps_offset(nbf) + (size_t)4 * nbf; }
inline size_t mixed_pdf_floats(int nbf) { return (pdf_region_bytes(nbf) + 3) / 4; }
// Byte offsets, within a chunk's scratch of `rows` slab rows, of the mixed form's planes that
// hold per-point values: Phi (float2 hi/lo), grad Phi hi words (3 float planes), their lo words
// (3 bf16 planes) and X / Z (float2 hi/lo); each plane is rows x 128 points.
struct MixedSlabOffsets {
    size_t phi, ghi, glo, x;
};
MixedSlabOffsets mixed_slab_offsets(int64_t rows);
// Tile widths the tcgen05 GEMMs are built for; `bn` below is one of them.
bool mixed_tile_supported(int bn);
void append_mixed_vtasks(int j, int n, int64_t s0, int64_t s1, int bn, std::vector<int> &tasks);
void build_mixed_schedule(const HostPlan &plan, const std::vector<int64_t> &chunk_t0,
                          const std::vector<int64_t> &chunk_t1, int bn, MixedSchedule &s);
void free_mixed_schedule(MixedSchedule &s);
void free_mixed_resident(MixedResident &r);
void free_mixed_ctx(MixedCtx &c);
// Driver entry point of the tensor-map encoder and kernel attributes (idempotent).
cudaError_t mixed_init(MixedCtx &c);
// Allocations of one in-flight mixed integration (call outside stream capture) ...
cudaError_t mixed_reserve(MixedCtx &c, const MixedSchedule &s, int nbf);
size_t mixed_reserve_bytes(const MixedSchedule &s, int nbf);
// ... and its per-call preparation on `st` (the P region, error word reset).
cudaError_t mixed_begin(MixedCtx &c, const double *P, int nbf, cudaStream_t st);
// Grouped chunks: each molecule's P region (mixed_pdf_floats(nbf) floats) and the reset of the
// error word, done by mixed_begin for a single molecule.
cudaError_t mixed_prepare_p(const double *P, float *pdf, int nbf, cudaStream_t st);
cudaError_t mixed_reset_error(MixedCtx &c, cudaStream_t st);
cudaError_t launch_mixed_chunk(const ChunkArgs &a, MixedCtx &c, MixedResident &r,
                               const MixedSchedule &s, int chunk_index, cudaStream_t st);
// Spin-unrestricted form: buffers for chunks of up to max_rows slab rows, the per-call
// preparation of P_a and P_b, and one chunk (a.Vacc receives W^j of spin a, Vacc_b spin b's).
cudaError_t mixed_reserve_uks(MixedCtx &c, int64_t max_rows, int nbf);
size_t mixed_reserve_uks_bytes(int64_t max_rows, int nbf);
cudaError_t mixed_begin_uks(MixedCtx &c, const double *Pa, const double *Pb, int nbf, cudaStream_t st);
cudaError_t launch_mixed_chunk_uks(const ChunkArgs &a, MixedCtx &c, MixedResident &r,
                                   const MixedSchedule &s, int chunk_index, double *Vacc_b, cudaStream_t st);
// Meta-GGA form (a.functional a meta-GGA): buffers for chunks of up to max_rows slab rows, and
// one chunk: X and Y^k = (d_k Phi) P^j on tcgen05, rho, grad rho, tau, the functional, Z and
// W^k, then the four V terms Z^T Phi + sum_k W^k^T d_k Phi into a.Vacc.
cudaError_t mixed_reserve_mgga(MixedCtx &c, int64_t max_rows);
cudaError_t launch_mixed_chunk_mgga(const ChunkArgs &a, MixedCtx &c, MixedResident &r,
                                    const MixedSchedule &s, int chunk_index, cudaStream_t st);
// Device error word of the mixed kernels (nonzero after a bounded wait expired).
cudaError_t mixed_read_error(MixedCtx &c, int *err, cudaStream_t st);

}  // namespace gbxc
