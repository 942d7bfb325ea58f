// horner_b.cu -- per-member Horner kernels for degrees 7..8 (see horner.cuh).
#include "horner.cuh"

namespace hwc {

const void *horner_kernel_b(int D, int which)
{
    switch (D) {
    case 7: return horner_pick<7>(which);
    case 8: return horner_pick<8>(which);
    default: return nullptr;
    }
}

}  // namespace hwc
