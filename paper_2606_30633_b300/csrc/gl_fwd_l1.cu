// k_forward instantiations with 1 lens-light component(s).
#include "gl_fwd_impl.cuh"

namespace gl {
GL_FWD_INST(, 1)
}  // namespace gl
