// k_grad / k_grad_multi instantiations with 0 lens-light component(s),
// exact-series deflection.
#include "gl_grad_impl.cuh"

namespace gl {
GL_GRAD_INST_S(, 0, false)
}  // namespace gl
