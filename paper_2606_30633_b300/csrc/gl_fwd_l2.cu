// k_forward instantiations with 2 lens-light component(s).
#include "gl_fwd_impl.cuh"

namespace gl {
GL_FWD_INST(, 2)
}  // namespace gl
