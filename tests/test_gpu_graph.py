"""A batched call captured into a CUDA graph and replayed: tinv_batch with device pointers, a
caller workspace and the problem table already in it enqueues kernels only, so a graph replay
must give the same vectors, bit for bit, as the direct call."""
import numpy as np
import pytest

from paper_1209_1910_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_batch_graph_replay_matches_direct_call():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_1910_gb300 import binding, build

    build.build()
    binding.load()
    dev = torch.device("cuda:0")
    sizes = [64, 210, 97, 420, 150, 21 * 12]
    probs = []
    for q, n in enumerate(sizes):
        d, e = inputs.glued_wilkinson(n // 21, 1e-10) if n % 21 == 0 else inputs.uniform(n, seed=70 + q)
        probs.append((d, e))
    ns, off_de, off_z = binding.pack_offsets([len(p[0]) for p in probs])
    M = int(ns.sum())
    D = np.zeros(M)
    E = np.zeros(M)
    for q, (d, e) in enumerate(probs):
        D[off_de[q]:off_de[q] + ns[q]] = d
        E[off_de[q]:off_de[q] + ns[q] - 1] = e
    td, te = torch.from_numpy(D).to(dev), torch.from_numpy(E).to(dev)
    tw = torch.zeros(M, dtype=torch.float64, device=dev)
    binding.bisect_batch_device(ns, off_de, td, te, tw)
    ws = torch.empty(binding.batch_workspace_size(ns), dtype=torch.uint8, device=dev)
    z_direct = torch.zeros(int((ns * ns).sum()), dtype=torch.float64, device=dev)
    z_graph = torch.zeros_like(z_direct)
    info = torch.zeros(len(ns), dtype=torch.int64, device=dev)
    # direct call: also writes the problem table into the workspace
    binding.tinv_batch_device(ns, off_de, off_z, td, te, tw, z_direct, info=info, workspace=ws)
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0] * len(ns)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            binding.tinv_batch_device(ns, off_de, off_z, td, te, tw, z_graph, info=info,
                                      workspace=ws, table_ready=1)
    for _ in range(2):
        z_graph.zero_()
        info.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert info.cpu().tolist() == [0] * len(ns)
        assert torch.equal(z_graph, z_direct)
