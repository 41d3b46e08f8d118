// Instantiations of the fused step for fp32 population storage.
#include "lbm_step.cuh"

namespace lbm {

void register_step_fp32(std::vector<StepVariant>& out)
{
    out.push_back({kFP32, 1, 4, &launch_step<kFP32, 1, 4>});
    out.push_back({kFP32, 1, 8, &launch_step<kFP32, 1, 8>});
    out.push_back({kFP32, 2, 4, &launch_step<kFP32, 2, 4>});
    out.push_back({kFP32, 2, 8, &launch_step<kFP32, 2, 8>});
    out.push_back({kFP32, 4, 4, &launch_step<kFP32, 4, 4>});
    out.push_back({kFP32, 4, 8, &launch_step<kFP32, 4, 8>});
}

}  // namespace lbm
