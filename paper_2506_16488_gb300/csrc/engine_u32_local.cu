// The persistent engine, the one-CTA (bucketed) kernel, for 32-bit tentative
// distances.
#include "engine_core.cuh"

namespace ppsp {

ppsp_status launch_engine_u32_local(const EngineArgs& a, int block_threads, u32 grid, cudaStream_t stream) {
    return launch_family<u32, true>(a, block_threads, grid, stream);
}

ppsp_status engine_occupancy_u32_local(int block_threads, u32 ring_cap, int* bpsm) {
    return occ_family<u32, true>(block_threads, ring_cap, bpsm);
}

}  // namespace ppsp

#ifdef PPSP_PHASE_CLOCKS
// Profiling builds only (the one-CTA 32-bit instances count): copy (and optionally clear) the 16 phase cycle totals.
extern "C" int ppsp_debug_phase_clocks(unsigned long long* out16, int clear) {
    cudaError_t e = cudaMemcpyFromSymbol(out16, ppsp::g_phase_clk, 16 * sizeof(unsigned long long));
    if (e == cudaSuccess && clear) {
        static const unsigned long long zero[16] = {0};
        e = cudaMemcpyToSymbol(ppsp::g_phase_clk, zero, sizeof(zero));
    }
    return (int)e;
}
#endif
