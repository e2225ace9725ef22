"""One rank of the replica path of bench.py on CPU (gloo), launched by test_replicas.py under
torch.distributed.run: prints this rank's instance fingerprint and the max over ranks."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import importlib.util  # noqa: E402

import torch  # noqa: E402

spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
bench = importlib.util.module_from_spec(spec)
spec.loader.exec_module(bench)

rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
torch.distributed.init_process_group(backend="gloo")
args = type("A", (), {"small": True})()
inst = bench.make_instance(args, rank)
value = 1.5 + rank                                 # a rank-dependent "step time"
mx = bench.max_over_ranks(value, world)
print(json.dumps({"rank": rank, "b0": float(inst["b"][0]), "n": inst["n"], "max": mx}), flush=True)
torch.distributed.barrier()
torch.distributed.destroy_process_group()
