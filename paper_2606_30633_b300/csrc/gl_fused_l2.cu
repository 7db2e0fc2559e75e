// k_grad_fused instantiations with 2 lens-light component(s): the gradient
// kernel that builds each row's surrogate table itself (a translation unit of
// its own: its dynamic shared memory is aligned for the tensor-core operands).
#include "gl_fused.cuh"

namespace gl {
GL_FUSED_INST(, 2)
}  // namespace gl
