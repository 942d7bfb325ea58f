// fan2_wa.cu -- two-level fan-out kernels for degrees 3..6 with the members
// weighted by their multiplicities among the samples of a sampled family (see
// fanout2.cuh).
#include "fanout2.cuh"

namespace hwc {

const void *fan2_kernel_wa(int D)
{
    switch (D) {
    case 3: return fan2_pick<3, true>();
    case 4: return fan2_pick<4, true>();
    case 5: return fan2_pick<5, true>();
    case 6: return fan2_pick<6, true>();
    default: return nullptr;
    }
}

}  // namespace hwc
