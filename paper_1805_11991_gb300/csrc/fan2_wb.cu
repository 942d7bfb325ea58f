// fan2_wb.cu -- two-level fan-out kernels for degrees 7..10 with the members
// weighted by their multiplicities among the samples of a sampled family (see
// fanout2.cuh).
#include "fanout2.cuh"

namespace hwc {

const void *fan2_kernel_wb(int D)
{
    switch (D) {
    case 7: return fan2_pick<7, true>();
    case 8: return fan2_pick<8, true>();
    case 9: return fan2_pick<9, true>();
    case 10: return fan2_pick<10, true>();
    default: return nullptr;
    }
}

}  // namespace hwc
