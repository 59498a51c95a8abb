// gb_persist_768.cu -- persistent_kernel instantiations with 768 threads per
// CTA: one CTA per SM at up to 80 registers a thread (1,024 threads allow 64).
#include "gb_kernels.h"
#include "gb_persist.cuh"

namespace gbk {

const void *persistent_ptr_768(int wheel, int bc)
{
    if (wheel != 13) return nullptr;
    switch (bc) {
        case 0: return (const void *)persistent_kernel<13, 768, 0>;
        case 6: return (const void *)persistent_kernel<13, 768, 6>;
        case 8: return (const void *)persistent_kernel<13, 768, 8>;
    }
    return nullptr;
}

}  // namespace gbk
