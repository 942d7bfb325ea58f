// horner_a.cu -- per-member Horner kernels for degrees 3..6 (see horner.cuh).
#include "horner.cuh"

namespace hwc {

const void *horner_kernel_a(int D, int which)
{
    switch (D) {
    case 3: return horner_pick<3>(which);
    case 4: return horner_pick<4>(which);
    case 5: return horner_pick<5>(which);
    case 6: return horner_pick<6>(which);
    default: return nullptr;
    }
}

}  // namespace hwc
