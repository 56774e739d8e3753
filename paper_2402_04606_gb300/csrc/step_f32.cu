// The persistent step kernel (step_impl.cuh) for float population storage,
// compiled on its own so that the storage kinds build in parallel.
#include "step_impl.cuh"

int launch_step_f32(const DevPool& P, const StepArgs& A, int grid, int threads, size_t smem, sbot_stream_t s) {
    return launch_step_s<float, float>(P, A, grid, threads, smem, (cudaStream_t)s);
}

int step_occupancy_f32(int B, int coll, int threads, size_t smem, size_t* static_smem) {
    return step_occupancy_s<float, float>(B, coll, threads, smem, static_smem);
}
