// The persistent engine, the one-CTA (bucketed) kernel, for 64-bit tentative
// distances.
#include "engine_core.cuh"

namespace ppsp {

ppsp_status launch_engine_u64_local(const EngineArgs& a, int block_threads, u32 grid, cudaStream_t stream) {
    return launch_family<u64, true>(a, block_threads, grid, stream);
}

ppsp_status engine_occupancy_u64_local(int block_threads, u32 ring_cap, int* bpsm) {
    return occ_family<u64, true>(block_threads, ring_cap, bpsm);
}

}  // namespace ppsp
