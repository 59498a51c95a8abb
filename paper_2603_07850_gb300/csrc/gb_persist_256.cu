// gb_persist_256.cu -- persistent_kernel instantiations with 256 threads per CTA.
#include "gb_kernels.h"
#include "gb_persist.cuh"

namespace gbk {

const void *persistent_ptr_256(int wheel, int bc)
{
    if (wheel == 13) {
        switch (bc) {
            case 0: return (const void *)persistent_kernel<13, 256, 0>;
            case 4: return (const void *)persistent_kernel<13, 256, 4>;
            case 6: return (const void *)persistent_kernel<13, 256, 6>;
            case 8: return (const void *)persistent_kernel<13, 256, 8>;
        }
    } else if (wheel == 7) {
        switch (bc) {
            case 0: return (const void *)persistent_kernel<7, 256, 0>;
            case 4: return (const void *)persistent_kernel<7, 256, 4>;
            case 8: return (const void *)persistent_kernel<7, 256, 8>;
        }
    }
    return nullptr;
}

}  // namespace gbk
