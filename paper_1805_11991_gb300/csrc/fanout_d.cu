// fanout_d.cu -- c_0 fan-out kernels for degree 7 (see fanout.cuh).
#include "fanout.cuh"

namespace hwc {

const void *fan_kernel_d(int D, int W, bool persistent)
{
    switch (D) {
    case 7: return W == 1 ? fan_pick<7, 1>(persistent) : fan_pick<7, 2>(persistent);
    default: return nullptr;
    }
}

}  // namespace hwc
