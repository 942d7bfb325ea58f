// horner_c.cu -- per-member Horner kernels for degrees 9..10 (see horner.cuh).
#include "horner.cuh"

namespace hwc {

const void *horner_kernel_c(int D, int which)
{
    switch (D) {
    case 9: return horner_pick<9>(which);
    case 10: return horner_pick<10>(which);
    default: return nullptr;
    }
}

}  // namespace hwc
