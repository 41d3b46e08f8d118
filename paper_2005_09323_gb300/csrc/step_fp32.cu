// Instantiations of the fused step for fp32 population storage.
#include "lbm_step.cuh"
#include "lbm_step_rows.cuh"
#include "lbm_step_tb.cuh"

namespace lbm {

// Failure-detection self test: one thread waits, with the same bounded loop as
// the step kernel, on an mbarrier that nothing arrives at; the wait runs out
// after `spins` polls and the status records it.
__global__ void bounded_wait_probe_kernel(long long spins, int32_t* status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(smem_addr(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    bool done = false;
    for (long long i = 0; i < spins && !done; ++i) done = mbar_try_wait(smem_addr(&bar), 0);
    *status = done ? 0 : LBM_ERR_TIMEOUT;
}


void register_step_fp32(std::vector<StepVariant>& out)
{
    out.push_back({kFP32, 1, 4, &launch_step<kFP32, 1, 4>, 0, nullptr});
    out.push_back({kFP32, 1, 8, &launch_step<kFP32, 1, 8>, 0, nullptr});
    out.push_back({kFP32, 2, 4, &launch_step<kFP32, 2, 4>, 0, nullptr});
    out.push_back({kFP32, 2, 8, &launch_step<kFP32, 2, 8>, 0, nullptr});
    out.push_back({kFP32, 4, 4, &launch_step<kFP32, 4, 4>, 0, nullptr});
    out.push_back({kFP32, 4, 8, &launch_step<kFP32, 4, 8>, 0, nullptr});
    out.push_back({kFP32, 4, kRowThreads / 32, &launch_rows<kFP32, 4>, 1, &rows_supported<kFP32, 4>});
    // several steps per launch from shared memory: the small calls of one AMS branch
    out.push_back({kFP32, 1, kTbThreads / 32, &launch_tb<kFP32>, 2, &tb_supported<kFP32>});
    out.back().multi = kTbHalo;
}

}  // namespace lbm

extern "C" int lbm_selftest_bounded_wait(int64_t spins, void* stream, int32_t* status)
{
    using namespace lbm;
    if (!status || spins < 1 || spins > (int64_t(1) << 30)) return fail(LBM_ERR_ARG, "lbm_selftest_bounded_wait: spins");
    int32_t* d = nullptr;
    LBM_CUDA(cudaMalloc(&d, sizeof(int32_t)));
    bounded_wait_probe_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>((long long)spins, d);
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaMemcpyAsync(status, d, sizeof(int32_t), cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream));
    if (err == cudaSuccess) err = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    cudaFree(d);
    if (err != cudaSuccess) return cuda_fail(err, "lbm_selftest_bounded_wait");
    count_launches(1);
    return LBM_OK;
}
