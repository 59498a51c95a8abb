// gb_persist_512.cu -- persistent_kernel instantiations with 512 threads per CTA.
#include "gb_kernels.h"
#include "gb_persist.cuh"

namespace gbk {

const void *persistent_ptr_512(int wheel, int bc)
{
    if (wheel == 13) {
        switch (bc) {
            case 0: return (const void *)persistent_kernel<13, 512, 0>;
            case 4: return (const void *)persistent_kernel<13, 512, 4>;
            case 6: return (const void *)persistent_kernel<13, 512, 6>;
            case 8: return (const void *)persistent_kernel<13, 512, 8>;
        }
    } else if (wheel == 7) {
        switch (bc) {
            case 0: return (const void *)persistent_kernel<7, 512, 0>;
            case 4: return (const void *)persistent_kernel<7, 512, 4>;
            case 8: return (const void *)persistent_kernel<7, 512, 8>;
        }
    }
    return nullptr;
}

// the per-n search in one loop, for launches without open-mask slots
const void *persistent_one_loop_ptr_512() { return (const void *)persistent_kernel<13, 512, 0, true>; }

const void *serve_ptr_512(int wheel, int bc)
{
    if (wheel == 13 && bc == 8) return (const void *)serve_kernel<13, 512, 8>;
    if (wheel == 13 && bc == 0) return (const void *)serve_kernel<13, 512, 0>;
    return nullptr;
}

}  // namespace gbk
