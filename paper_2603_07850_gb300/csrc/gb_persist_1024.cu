// gb_persist_1024.cu -- persistent_kernel instantiations with 1024 threads per CTA.
#include "gb_kernels.h"
#include "gb_persist.cuh"

namespace gbk {

const void *persistent_ptr_1024(int wheel, int bc)
{
    if (wheel == 13) {
        switch (bc) {
            case 0: return (const void *)persistent_kernel<13, 1024, 0>;
            case 4: return (const void *)persistent_kernel<13, 1024, 4>;
            case 6: return (const void *)persistent_kernel<13, 1024, 6>;
            case 8: return (const void *)persistent_kernel<13, 1024, 8>;
        }
    } else if (wheel == 7) {
        switch (bc) {
            case 0: return (const void *)persistent_kernel<7, 1024, 0>;
            case 4: return (const void *)persistent_kernel<7, 1024, 4>;
            case 8: return (const void *)persistent_kernel<7, 1024, 8>;
        }
    }
    return nullptr;
}

const void *serve_ptr_1024(int wheel, int bc)
{
    if (wheel == 13 && bc == 8) return (const void *)serve_kernel<13, 1024, 8>;
    if (wheel == 13 && bc == 6) return (const void *)serve_kernel<13, 1024, 6>;
    if (wheel == 13 && bc == 4) return (const void *)serve_kernel<13, 1024, 4>;
    if (wheel == 13 && bc == 0) return (const void *)serve_kernel<13, 1024, 0>;
    return nullptr;
}

}  // namespace gbk
