// fanout_b.cu -- c_0 fan-out kernels for degree 5 (see fanout.cuh).
#include "fanout.cuh"

namespace hwc {

const void *fan_kernel_b(int D, int W, bool persistent)
{
    switch (D) {
    case 5: return W == 1 ? fan_pick<5, 1>(persistent) : fan_pick<5, 2>(persistent);
    default: return nullptr;
    }
}

}  // namespace hwc
