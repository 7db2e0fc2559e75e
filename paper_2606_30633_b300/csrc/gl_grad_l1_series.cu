// k_grad / k_grad_multi instantiations with 1 lens-light component(s),
// exact-series deflection.
#include "gl_grad_impl.cuh"

namespace gl {
GL_GRAD_INST_S(, 1, false)
}  // namespace gl
