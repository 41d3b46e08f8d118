// Instantiations of the fused step for bf16 population storage.
#include "lbm_step.cuh"

namespace lbm {

void register_step_bf16(std::vector<StepVariant>& out)
{
    out.push_back({kBF16, 2, 4, &launch_step<kBF16, 2, 4>});
    out.push_back({kBF16, 2, 8, &launch_step<kBF16, 2, 8>});
    out.push_back({kBF16, 4, 4, &launch_step<kBF16, 4, 4>});
    out.push_back({kBF16, 4, 8, &launch_step<kBF16, 4, 8>});
    out.push_back({kBF16, 8, 4, &launch_step<kBF16, 8, 4>});
    out.push_back({kBF16, 8, 8, &launch_step<kBF16, 8, 8>});
}

}  // namespace lbm
