"""Per-mechanism specialised kernels (stev_spec_compile_check): the
mixed-precision solver source compiles with NVRTC for sm_103a with the
mechanism's sizes as constants, for every kernel variant the library
selects (lane groups of 8, 16 and 32, the network kernel, global rate laws,
the unrolled N = 13 window and the run-time one).  Compilation only: no GPU
is needed; the GPU tests run the compiled kernels against the generic ones."""
import pytest

from paper_1905_09395_b300 import binding


@pytest.mark.parametrize("S,R,Rrev,general,G,N,net", [
    (32, 150, 150, False, 32, 13, False),   # the 32/150 workload
    (32, 150, 150, False, 32, 13, True),    # ... with the thermo network
    (8, 20, 20, False, 8, 13, False),       # the 8/20 mechanism, 4 cells per warp
    (8, 20, 20, False, 8, 13, True),        # ... with the network, 4 cells per warp
    (6, 2, 1, True, 8, 13, True),           # BFER with the network
    (53, 325, 325, False, 32, 13, False),   # 53/325, two species per lane
    (6, 2, 1, True, 8, 13, False),          # BFER: real orders and stoichiometry
    (16, 40, 40, False, 16, 9, False),      # a run-time window length
])
def test_specialised_kernel_compiles(S, R, Rrev, general, G, N, net):
    binding.spec_compile_check(S, R, Rrev, general=general, lanes_per_cell=G, dft_n=N,
                               network=net)


def test_bad_sizes_are_rejected():
    with pytest.raises(binding.StevError):
        binding.spec_compile_check(65, 10, 10)
    with pytest.raises(binding.StevError):
        binding.spec_compile_check(32, 150, 150, lanes_per_cell=4, network=True)
