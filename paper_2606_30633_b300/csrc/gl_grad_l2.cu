// k_grad instantiations with 2 lens-light component(s).
#include "gl_grad_impl.cuh"

namespace gl {
GL_GRAD_INST(, 2)
}  // namespace gl
