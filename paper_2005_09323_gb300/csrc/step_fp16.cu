// Instantiations of the fused step for fp16 population storage.
#include "lbm_step.cuh"

namespace lbm {

void register_step_fp16(std::vector<StepVariant>& out)
{
    out.push_back({kFP16, 2, 4, &launch_step<kFP16, 2, 4>});
    out.push_back({kFP16, 2, 8, &launch_step<kFP16, 2, 8>});
    out.push_back({kFP16, 4, 4, &launch_step<kFP16, 4, 4>});
    out.push_back({kFP16, 4, 8, &launch_step<kFP16, 4, 8>});
    out.push_back({kFP16, 8, 4, &launch_step<kFP16, 8, 4>});
    out.push_back({kFP16, 8, 8, &launch_step<kFP16, 8, 8>});
}

}  // namespace lbm
