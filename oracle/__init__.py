"""Plain FP64 CPU oracle for PDHG with online preconditioning (Lu & Zhang,
"Enhanced PDHG for Linear Programming with Online Preconditioning").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` use it.  It shares no code with the
CUDA library; the two meet only through the seeded generators in ``lpgen``.

Modules
-------
* :mod:`oracle.pdhg` -- the method, step by step, in numpy float64.
* :mod:`oracle.vertices` -- brute-force vertex enumeration for tiny LPs.

Parity status of each function is stated in its docstring ("pinned by ...");
every public function has a pin.
"""
from .pdhg import (  # noqa: F401
    Options,
    Scaled,
    State,
    Result,
    scale_problem,
    ruiz_equilibrate,
    pock_chambolle_rescale,
    l2_norm_rescale,
    power_spectral_norm,
    initial_state,
    primal_half_step,
    dual_half_step,
    online_gradients,
    ogd_update,
    step_size_limit,
    attempt,
    kkt,
    check,
    solve,
    unscale,
    lagrangian,
)
from .vertices import enumerate_vertices  # noqa: F401
