// k_grad instantiations with 1 lens-light component(s).
#include "gl_grad_impl.cuh"

namespace gl {
GL_GRAD_INST(, 1)
}  // namespace gl
