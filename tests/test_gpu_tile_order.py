"""gs_tile_order against its definition: tiles by decreasing list length
(clamped to 65535), ties by tile id.  Both of its paths: the one-launch
counting rank (up to 12288 tiles) and the radix sort (more tiles), with many
ties, empty tiles, lengths past the clamp and the sizes at the switch."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_02121_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _expected(ranges):
    length = np.minimum(np.maximum(ranges[:, 1] - ranges[:, 0], 0), 65535)
    return np.lexsort((np.arange(len(ranges)), 65535 - length))


@pytest.mark.parametrize("T", [1, 3, 31, 1000, 8160, 12287, 12288, 12289, 30000])
def test_tile_order_matches_the_definition(T):
    rng = np.random.default_rng(T)
    # lengths drawn from few values (many ties), some empty, some past the 65535 clamp
    length = rng.choice([0, 1, 7, 7, 443, 443, 2000, 70000, 65535, 65536], size=T)
    start = np.cumsum(np.concatenate([[0], length[:-1]])).astype(np.int64) % (1 << 30)
    ranges = np.stack([start, start + length], axis=1).astype(np.int32)
    tr = torch.as_tensor(ranges, device="cuda")
    ws = torch.empty(B.gs_tile_order_workspace_size(T), dtype=torch.uint8, device="cuda")
    order = torch.full((T,), -1, dtype=torch.int32, device="cuda")
    B.gs_tile_order(tr, T, ws, order)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(order.cpu().numpy(), _expected(ranges))
