// Mixed-precision form: float32 collocation, split-bf16x3 tcgen05 contractions
// with float32 accumulation in tensor memory, float64 weights, functional tail
// and accumulation.
#pragma once

#include <cstdint>
#include <vector>

#include "internal.h"

namespace gbxc {

size_t fp64_row_bytes();
void append_fp64_vtasks(int j, int n, int64_t s0, int64_t s1, std::vector<int> &tasks);

// Per-context state of the mixed form (tensor-map encoder, P split buffers).
struct MixedCtx {
    void *encode_fn = nullptr;         // cuTensorMapEncodeTiled from the driver
    uint16_t *Phl = nullptr;           // gathered P^j blocks, bf16 hi/lo
    size_t phl_cap = 0;
};
// Per-molecule resident state of the mixed form.
struct MixedResident {
    int dummy = 0;
};
// Per-schedule state of the mixed form (P^j gather layout).
struct MixedSchedule {
    int64_t *d_pofs = nullptr;         // per batch: element offset of its packed P^j
    int64_t ptotal = 0;                // elements of all packed P^j
    int b0 = 0, b1 = 0;
};

size_t mixed_row_bytes();
void append_mixed_vtasks(int j, int n, int64_t s0, int64_t s1, std::vector<int> &tasks);
void build_mixed_schedule(const HostPlan &plan, int nbf, int b0, int b1, MixedSchedule &s);
void free_mixed_schedule(MixedSchedule &s);
void free_mixed_resident(MixedResident &r);
void free_mixed_ctx(MixedCtx &c);
cudaError_t mixed_prepare(MixedCtx &c, MixedResident &r, const MixedSchedule &s, const double *P,
                          int nbf, cudaStream_t st);
cudaError_t launch_mixed_chunk(const ChunkArgs &a, MixedCtx &c, MixedResident &r,
                               const MixedSchedule &s, cudaStream_t st);

}  // namespace gbxc
