// Tile selection for a plan.
#include "plan_impl.h"

namespace stencil {

int tune_plan(Plan *p, const stencil_desc *d)
{
    (void)p;
    (void)d;
    return fail(STENCIL_EUNSUPPORTED, "tile selection not built yet");
}

}  // namespace stencil
