// Engine dispatch by distance width, and the small kernels of a plan run
// (potential evaluation, result scatter).
#include "engine_core.cuh"

namespace ppsp {

// instantiated in engine_{u32,u64}{,_local}.cu
ppsp_status launch_engine_u32(const EngineArgs& a, int block_threads, u32 grid, cudaStream_t stream);
ppsp_status launch_engine_u64(const EngineArgs& a, int block_threads, u32 grid, cudaStream_t stream);
ppsp_status launch_engine_u32_local(const EngineArgs& a, int block_threads, u32 grid, cudaStream_t stream);
ppsp_status launch_engine_u64_local(const EngineArgs& a, int block_threads, u32 grid, cudaStream_t stream);
ppsp_status engine_occupancy_u32(int block_threads, u32 ring_cap, int* bpsm);
ppsp_status engine_occupancy_u64(int block_threads, u32 ring_cap, int* bpsm);
ppsp_status engine_occupancy_u32_local(int block_threads, u32 ring_cap, int* bpsm);
ppsp_status engine_occupancy_u64_local(int block_threads, u32 ring_cap, int* bpsm);

ppsp_status launch_engine(const EngineArgs& a, int dist_bits, int block_threads, u32 grid,
                          cudaStream_t stream, bool local_only) {
    if (dist_bits == 32)
        return local_only ? launch_engine_u32_local(a, block_threads, grid, stream)
                          : launch_engine_u32(a, block_threads, grid, stream);
    return local_only ? launch_engine_u64_local(a, block_threads, grid, stream)
                      : launch_engine_u64(a, block_threads, grid, stream);
}

ppsp_status engine_occupancy(int dist_bits, int block_threads, int* blocks_per_sm, int* sms, bool local_only,
                             u32 ring_cap) {
    int dev = 0;
    PPSP_CUDA_TRY(cudaGetDevice(&dev));
    PPSP_CUDA_TRY(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
    if (dist_bits == 32)
        return local_only ? engine_occupancy_u32_local(block_threads, ring_cap, blocks_per_sm)
                          : engine_occupancy_u32(block_threads, ring_cap, blocks_per_sm);
    return local_only ? engine_occupancy_u64_local(block_threads, ring_cap, blocks_per_sm)
                      : engine_occupancy_u64(block_threads, ring_cap, blocks_per_sm);
}

// ---- potential evaluation (for checks against the oracle) ----
__global__ void potential_eval_kernel(GraphDev g, u32 anchor, const u32* verts, u64 count, i64* out) {
    u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    u32 v = verts[k];
    out[k] = (v < g.n) ? pot_h(g.pc[anchor], g.pc[v], g.pot_shift) : -1;
}

ppsp_status launch_potential_eval(const GraphDev& g, u32 anchor, const u32* d_verts, u64 count,
                                  i64* d_out, cudaStream_t stream) {
    if (count == 0) return PPSP_OK;
    u32 blocks = (u32)((count + 255) / 256);
    potential_eval_kernel<<<blocks, 256, 0, stream>>>(g, anchor, d_verts, count, d_out);
    PPSP_CUDA_TRY(cudaGetLastError());
    return PPSP_OK;
}

__global__ void scatter_kernel(const u32* map, const u64* mu, u64 k, u64* out) {
    u64 q = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= k) return;
    u32 m = map[q];
    out[q] = (m == NONE) ? 0ull : mu[m];
}

ppsp_status launch_scatter(const u32* d_map, const u64* d_mu, u64 k, u64* d_out, cudaStream_t s) {
    if (k == 0) return PPSP_OK;
    u32 blocks = (u32)((k + 255) / 256);
    scatter_kernel<<<blocks, 256, 0, s>>>(d_map, d_mu, k, d_out);
    PPSP_CUDA_TRY(cudaGetLastError());
    return PPSP_OK;
}

}  // namespace ppsp

