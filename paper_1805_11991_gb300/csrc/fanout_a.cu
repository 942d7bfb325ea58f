// fanout_a.cu -- c_0 fan-out kernels for degrees 3, 4 (see fanout.cuh).
#include "fanout.cuh"

namespace hwc {

const void *fan_kernel_a(int D, int W, bool persistent)
{
    switch (D) {
    case 3: return W == 1 ? fan_pick<3, 1>(persistent) : fan_pick<3, 2>(persistent);
    case 4: return W == 1 ? fan_pick<4, 1>(persistent) : fan_pick<4, 2>(persistent);
    default: return nullptr;
    }
}

}  // namespace hwc
