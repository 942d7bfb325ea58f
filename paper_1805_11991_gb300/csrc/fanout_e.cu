// fanout_e.cu -- c_0 fan-out kernels for degrees 9, 10 (see fanout.cuh).
#include "fanout.cuh"

namespace hwc {

const void *fan_kernel_e(int D, int W, bool persistent)
{
    switch (D) {
    case 9: return W == 1 ? fan_pick<9, 1>(persistent) : nullptr;   // q >= 32: q^4 > HWC_MAX_Q
    case 10: return W == 1 ? fan_pick<10, 1>(persistent) : nullptr;   // q >= 32: q^4 > HWC_MAX_Q
    default: return nullptr;
    }
}

}  // namespace hwc
