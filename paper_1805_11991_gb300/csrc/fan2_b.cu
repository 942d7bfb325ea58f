// fan2_b.cu -- two-level fan-out kernels for degrees 7..10 (see fanout2.cuh).
#include "fanout2.cuh"

namespace hwc {

const void *fan2_kernel_b(int D)
{
    switch (D) {
    case 7: return fan2_pick<7>();
    case 8: return fan2_pick<8>();
    case 9: return fan2_pick<9>();
    case 10: return fan2_pick<10>();
    default: return nullptr;
    }
}

}  // namespace hwc
