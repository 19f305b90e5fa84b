// Mixed-precision form (placeholder until the tensor-core kernels land).
#include "mixed.h"

namespace gbxc {

size_t mixed_row_bytes() { return (size_t)TILE * 16; }
void append_mixed_vtasks(int, int, int64_t, int64_t, std::vector<int> &) {}
void build_mixed_schedule(const HostPlan &, int, int b0, int b1, MixedSchedule &s) {
    s.b0 = b0;
    s.b1 = b1;
}
void free_mixed_schedule(MixedSchedule &s) { s = MixedSchedule{}; }
void free_mixed_resident(MixedResident &r) { r = MixedResident{}; }
void free_mixed_ctx(MixedCtx &c) { c = MixedCtx{}; }
cudaError_t mixed_prepare(MixedCtx &, MixedResident &, const MixedSchedule &, const double *, int,
                          cudaStream_t) {
    return cudaErrorNotSupported;
}
cudaError_t launch_mixed_chunk(const ChunkArgs &, MixedCtx &, MixedResident &,
                               const MixedSchedule &, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace gbxc
