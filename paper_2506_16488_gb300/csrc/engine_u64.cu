// The persistent engine, the general kernel (queue / bitmap path and one-CTA path), for 64-bit tentative
// distances.
#include "engine_core.cuh"

namespace ppsp {

ppsp_status launch_engine_u64(const EngineArgs& a, int block_threads, u32 grid, cudaStream_t stream) {
    return launch_family<u64, false>(a, block_threads, grid, stream);
}

ppsp_status engine_occupancy_u64(int block_threads, u32 ring_cap, int* bpsm) {
    return occ_family<u64, false>(block_threads, ring_cap, bpsm);
}

}  // namespace ppsp
