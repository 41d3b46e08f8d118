// Instantiations of the fused step for fp16 population storage.
#include "lbm_step.cuh"
#include "lbm_step_rows.cuh"
#include "lbm_step_tb.cuh"

namespace lbm {

void register_step_fp16(std::vector<StepVariant>& out)
{
    out.push_back({kFP16, 2, 4, &launch_step<kFP16, 2, 4>, 0, nullptr});
    out.push_back({kFP16, 2, 8, &launch_step<kFP16, 2, 8>, 0, nullptr});
    out.push_back({kFP16, 4, 4, &launch_step<kFP16, 4, 4>, 0, nullptr});
    out.push_back({kFP16, 4, 8, &launch_step<kFP16, 4, 8>, 0, nullptr});
    out.push_back({kFP16, 8, 4, &launch_step<kFP16, 8, 4>, 0, nullptr});
    out.push_back({kFP16, 8, 8, &launch_step<kFP16, 8, 8>, 0, nullptr});
    out.push_back({kFP16, 4, kRowThreads / 32, &launch_rows<kFP16, 4>, 1, &rows_supported<kFP16, 4>});
    out.push_back({kFP16, 8, kRowThreads / 32, &launch_rows<kFP16, 8>, 1, &rows_supported<kFP16, 8>});
    // several steps per launch from shared memory: the small calls of one AMS branch
    out.push_back({kFP16, 1, kTbThreads / 32, &launch_tb<kFP16>, 2, &tb_supported<kFP16>});
    out.back().multi = kTbHalo;
}

}  // namespace lbm
