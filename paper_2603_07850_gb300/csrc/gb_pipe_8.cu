// gb_pipe_8.cu -- pipelined persistent kernel instantiations with 8 window-building warps.
#include "gb_kernels.h"
#include "gb_persist.cuh"

namespace gbk {

const void *pipe_ptr_8(int nt, int bc)
{
    if (nt == 1024) {                    // 8 building + 24 searching warps
        switch (bc) {
            case 0: return (const void *)pipe_kernel<13, 8, 24, 0>;
            case 4: return (const void *)pipe_kernel<13, 8, 24, 4>;
            case 6: return (const void *)pipe_kernel<13, 8, 24, 6>;
            case 8: return (const void *)pipe_kernel<13, 8, 24, 8>;
        }
    } else if (nt == 768) {              // 8 building + 16 searching warps, 80 registers a thread
        switch (bc) {
            case 6: return (const void *)pipe_kernel<13, 8, 16, 6>;
        }
    }
    return nullptr;
}

}  // namespace gbk
