// gb_pipe_16.cu -- pipelined persistent kernel instantiations with 12 or 16
// window-building warps.
#include "gb_kernels.h"
#include "gb_persist.cuh"

namespace gbk {

const void *pipe_ptr_16(int np, int nt, int bc)
{
    if (np == 16 && nt == 1024) {        // 16 building + 16 searching warps
        switch (bc) {
            case 0: return (const void *)pipe_kernel<13, 16, 16, 0>;
            case 4: return (const void *)pipe_kernel<13, 16, 16, 4>;
            case 6: return (const void *)pipe_kernel<13, 16, 16, 6>;
            case 8: return (const void *)pipe_kernel<13, 16, 16, 8>;
        }
    } else if (np == 12 && nt == 1024) { // 12 building + 20 searching warps
        switch (bc) {
            case 6: return (const void *)pipe_kernel<13, 12, 20, 6>;
        }
    }
    return nullptr;
}

}  // namespace gbk
