// k_grad instantiations with 0 lens-light component(s).
#include "gl_grad_impl.cuh"

namespace gl {
GL_GRAD_INST(, 0)
}  // namespace gl
