"""Host-side checks of the Python binding's autograd plumbing with a stand-in
renderer (no GPU, no library call): `render` passes every parameter tensor
the scene holds, the optional ones included, and returns their gradients."""
import torch

from paper_2604_24994_gb300 import api


class FakeScene:
    def __init__(self, params):
        self.params = params


class FakeRenderer:
    """Records what the binding hands over; 'renders' rgb = sum of every
    parameter's sum, so each gradient is all ones times the upstream sum."""
    generation = 0

    def __init__(self):
        self.seen_fwd = None
        self.seen_bwd = None

    def bin(self, scene, pd):
        return 0

    def render_fwd(self, scene, pd):
        self.seen_fwd = tuple(pd)
        tot = sum(v.sum() for v in pd.values())
        rgb = torch.full((4, 3), float(tot))
        return rgb, torch.ones(4), torch.zeros(4, dtype=torch.int32)

    def backward(self, scene, g_rgb, g_T, T, last, pd):
        self.seen_bwd = tuple(pd)
        return {k: torch.full_like(v, float(g_rgb.sum())) for k, v in pd.items()}


def params(extra=()):
    p = {k: torch.rand(3, requires_grad=True) for k in api.PARAMS}
    for k in extra:
        p[k] = torch.rand(5, requires_grad=True)
    return p


def test_render_passes_the_base_parameters():
    r = FakeRenderer()
    p = params()
    rgb, T = api.render(r, FakeScene(p))
    rgb.sum().backward()
    assert r.seen_fwd == api.PARAMS and r.seen_bwd == api.PARAMS
    for k in api.PARAMS:
        assert torch.all(p[k].grad == 12.0)


def test_render_passes_the_optional_parameters():
    r = FakeRenderer()
    p = params(("disp", "sv"))
    rgb, T = api.render(r, FakeScene(p))
    (2 * rgb).sum().backward()
    assert r.seen_fwd == api.PARAMS + ("disp", "sv")
    for k in api.PARAMS + ("disp", "sv"):
        assert torch.all(p[k].grad == 24.0), k
