"""Host-side checks of the Python binding (CPU, nothing launches): tensors
must be CUDA float32 and contiguous, shapes must match the grid, the variant
table resolves to the paper's channel counts, and the binding has no CPU
fallback."""
import pytest
import torch

from paper_2505_21319_gb300 import api


def test_cpu_tensors_are_rejected_before_any_launch():
    p = torch.zeros(8 ** 3 * 13)
    q = torch.zeros(10, 3)
    with pytest.raises(TypeError):
        api.efunc_forward(p, q)
    with pytest.raises(TypeError):
        api.efunc_backward(p, q, torch.zeros(10))
    with pytest.raises(TypeError):
        api.efunc_mean_shift_init(p, torch.zeros(5, 3))
    with pytest.raises(TypeError):
        api.efunc_variant_forward("G-6", torch.zeros(8 ** 3 * 5), q)
    with pytest.raises(TypeError):
        api.efunc_cosine_forward(2, torch.zeros(2 * 8 ** 3 * 5), q)
    assert api.launch_count() == 0


def test_parameter_sizes_must_match_a_grid():
    with pytest.raises(ValueError):
        api.resolution_of(torch.zeros(1000))
    assert api.resolution_of(torch.zeros(32 ** 3 * 13)) == 32
    with pytest.raises(ValueError):
        api._variant_resolution(torch.zeros(8 ** 3 * 5 + 1), 5)


def test_variant_names_resolve_to_the_table():
    assert api.variant_channels("G-6") == 5
    assert api.variant_channels((3, 1, 1)) == 13
    with pytest.raises(KeyError):
        api.make_variant("G-9")
    with pytest.raises(ValueError):
        api.variant_channels((4, 1, 1))


def test_status_codes_raise_with_their_description():
    from paper_2505_21319_gb300 import _binding as B
    with pytest.raises(B.EfuncError, match="invalid argument"):
        B.check("efunc_forward", 1)
    B.check("efunc_forward", 0)
    # a CUDA failure names the CUDA error behind it (none recorded here)
    with pytest.raises(B.EfuncError, match="CUDA runtime error: cudaSuccess") as info:
        B.check("efunc_fit", 2)
    assert info.value.cuda_error == 0 and info.value.code == 2


def test_graph_fit_is_the_pipelined_schedule():
    p = torch.zeros(8 ** 3 * 13)
    with pytest.raises(ValueError):
        api.efunc_fit(p, p, p, torch.zeros(10, 4), steps=1, graph=True, pipelined=False)
    assert api.launch_count() == 0
