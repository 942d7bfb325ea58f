// cls_a.cu -- class-sharing count kernels for degrees 3..6 (see classes.cuh).
#include "classes.cuh"

namespace hwc {

const void *cls_kernel_a(int D, int which)
{
    switch (D) {
    case 3: return cls_pick<3>(which);
    case 4: return cls_pick<4>(which);
    case 5: return cls_pick<5>(which);
    case 6: return cls_pick<6>(which);
    default: return nullptr;
    }
}

}  // namespace hwc
