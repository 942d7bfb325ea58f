// fanout_f.cu -- c_0 fan-out kernels for degree 8 (see fanout.cuh).
#include "fanout.cuh"

namespace hwc {

const void *fan_kernel_f(int D, int W, bool persistent)
{
    switch (D) {
    case 8: return W == 1 ? fan_pick<8, 1>(persistent) : fan_pick<8, 2>(persistent);
    default: return nullptr;
    }
}

}  // namespace hwc
