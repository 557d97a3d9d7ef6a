"""GB300 (sm_103a) implementation of the pulse-noise many-spin time step of
D. A. Garanin, "Pulse-noise approach for classical spin systems"
(arXiv:1610.04914).

The compute path is the CUDA library ``libspinpulse.so`` behind the C-ABI of
include/spinpulse.h; this package only marshals arguments to it.  Build the
library with ``paper_1610_04914_gb300.build.build()``.
"""
from ._binding import (HEUN, RK2_MIDPOINT, RK4, RK5_BUTCHER, SPIN_ENONFINITE, SPIN_OK,  # noqa: F401
                       SPIN_WARN_APPLICABILITY, SpinError, load)
from .lattice import (EscapeReplicas, Lattice, Params, SingleSpins, SpinRunFn, spin_backward, spin_backward_workspace_size,  # noqa: F401
                      spin_get_step, spin_lattice_create, spin_record_begin, spin_record_end,
                      spin_record_store_size,
                      spin_lattice_destroy, spin_metropolis_color, spin_metropolis_sweeps, spin_noise_draw, spin_observables,
                      spin_observables_noalloc, spin_samples,
                      spin_set_step, spin_step_pulse, spin_workspace_size)
from .batch import Batch, spin_batch_offsets, spin_batch_tile_rows, spin_batch_workspace_size  # noqa: F401,E402
