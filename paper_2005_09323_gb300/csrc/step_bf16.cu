// Instantiations of the fused step for bf16 population storage.
#include "lbm_step.cuh"
#include "lbm_step_rows.cuh"
#include "lbm_step_tb.cuh"

namespace lbm {

void register_step_bf16(std::vector<StepVariant>& out)
{
    out.push_back({kBF16, 2, 4, &launch_step<kBF16, 2, 4>, 0, nullptr});
    out.push_back({kBF16, 2, 8, &launch_step<kBF16, 2, 8>, 0, nullptr});
    out.push_back({kBF16, 4, 4, &launch_step<kBF16, 4, 4>, 0, nullptr});
    out.push_back({kBF16, 4, 8, &launch_step<kBF16, 4, 8>, 0, nullptr});
    out.push_back({kBF16, 8, 4, &launch_step<kBF16, 8, 4>, 0, nullptr});
    out.push_back({kBF16, 8, 8, &launch_step<kBF16, 8, 8>, 0, nullptr});
    out.push_back({kBF16, 4, kRowThreads / 32, &launch_rows<kBF16, 4>, 1, &rows_supported<kBF16, 4>});
    out.push_back({kBF16, 8, kRowThreads / 32, &launch_rows<kBF16, 8>, 1, &rows_supported<kBF16, 8>});
    // several steps per launch from shared memory: the small calls of one AMS branch
    out.push_back({kBF16, 1, kTbThreads / 32, &launch_tb<kBF16>, 2, &tb_supported<kBF16>});
    out.back().multi = kTbHalo;
}

}  // namespace lbm
