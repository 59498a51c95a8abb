// gb_persist_512.cu -- persistent_kernel instantiations with 512 threads per CTA.
#include "gb_kernels.h"
#include "gb_persist.cuh"

namespace gbk {

const void *persistent_ptr_512(int wheel, int bc)
{
    if (wheel == 13) {
        switch (bc) {
            case 0: return (const void *)persistent_kernel<13, 512, 0>;
            case 2: return (const void *)persistent_kernel<13, 512, 2>;
            case 3: return (const void *)persistent_kernel<13, 512, 3>;
            case 4: return (const void *)persistent_kernel<13, 512, 4>;
        }
    } else if (wheel == 7) {
        switch (bc) {
            case 0: return (const void *)persistent_kernel<7, 512, 0>;
            case 3: return (const void *)persistent_kernel<7, 512, 3>;
            case 4: return (const void *)persistent_kernel<7, 512, 4>;
        }
    }
    return nullptr;
}

const void *serve_ptr_512(int wheel, int bc)
{
    if (wheel == 13 && bc == 3) return (const void *)serve_kernel<13, 512, 3>;
    if (wheel == 13 && bc == 0) return (const void *)serve_kernel<13, 512, 0>;
    return nullptr;
}

}  // namespace gbk
