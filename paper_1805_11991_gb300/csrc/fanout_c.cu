// fanout_c.cu -- c_0 fan-out kernels for degree 6 (see fanout.cuh).
#include "fanout.cuh"

namespace hwc {

const void *fan_kernel_c(int D, int W, bool persistent)
{
    switch (D) {
    case 6: return W == 1 ? fan_pick<6, 1>(persistent) : fan_pick<6, 2>(persistent);
    default: return nullptr;
    }
}

}  // namespace hwc
