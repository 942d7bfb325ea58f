// fan2_a.cu -- two-level fan-out kernels for degrees 3..6 (see fanout2.cuh).
#include "fanout2.cuh"

namespace hwc {

const void *fan2_kernel_a(int D)
{
    switch (D) {
    case 3: return fan2_pick<3>();
    case 4: return fan2_pick<4>();
    case 5: return fan2_pick<5>();
    case 6: return fan2_pick<6>();
    default: return nullptr;
    }
}

}  // namespace hwc
