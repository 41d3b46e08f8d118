// Open-channel instantiations of the fused step for 16-bit population storage
// (Sec. 2: grid of bars, sponge, inlet and outlet columns); the row-staged
// variants have none.
#include "lbm_step.cuh"

namespace lbm {

template <int S>
void register_open_16(std::vector<StepVariant>& v)
{
    for (auto& s : v) {
        if (s.storage != S || s.kind != 0) continue;
        if (s.vec == 2 && s.warps == 8) s.launch_open = &launch_step_open<S, 2, 8>;
        if (s.vec == 4 && s.warps == 4) s.launch_open = &launch_step_open<S, 4, 4>;
        if (s.vec == 8 && s.warps == 4) s.launch_open = &launch_step_open<S, 8, 4>;
        if (s.vec == 8 && s.warps == 8) s.launch_open = &launch_step_open<S, 8, 8>;
    }
}

void register_open_fp16(std::vector<StepVariant>& v) { register_open_16<kFP16>(v); }
void register_open_bf16(std::vector<StepVariant>& v) { register_open_16<kBF16>(v); }

}  // namespace lbm
