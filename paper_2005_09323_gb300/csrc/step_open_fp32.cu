// Open-channel instantiations of the fused step for fp32 population storage
// (Sec. 2: grid of bars, sponge, inlet and outlet columns); the row-staged
// variant has none.
#include "lbm_step.cuh"

namespace lbm {

void register_open_fp32(std::vector<StepVariant>& v)
{
    for (auto& s : v) {
        if (s.storage != kFP32 || s.kind != 0) continue;
        if (s.vec == 1 && s.warps == 8) s.launch_open = &launch_step_open<kFP32, 1, 8>;
        if (s.vec == 2 && s.warps == 8) s.launch_open = &launch_step_open<kFP32, 2, 8>;
        if (s.vec == 4 && s.warps == 4) s.launch_open = &launch_step_open<kFP32, 4, 4>;
        if (s.vec == 4 && s.warps == 8) s.launch_open = &launch_step_open<kFP32, 4, 8>;
    }
}

}  // namespace lbm
