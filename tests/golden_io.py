"""Reader for the hand-worked fixtures under tests/golden/."""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field
from typing import Dict, List, Set, Tuple

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@dataclass
class Fixture:
    name: str
    n: int = 0
    concepts: Dict[int, Set[int]] = field(default_factory=dict)
    roles: Dict[int, List[Tuple[int, int]]] = field(default_factory=dict)
    props: Dict[int, Dict[int, float]] = field(default_factory=dict)
    pos: Set[int] = field(default_factory=set)
    neg: Set[int] = field(default_factory=set)
    queries: List[Tuple[str, Set[int], Tuple[int, int, int, int]]] = field(default_factory=list)

    def concept_list(self):
        return [self.concepts.get(i, set()) for i in range(max(self.concepts, default=-1) + 1)]

    def role_list(self):
        return [self.roles.get(i, []) for i in range(max(self.roles, default=-1) + 1)]

    def prop_rows(self):
        rows = []
        for p in range(max(self.props, default=-1) + 1):
            d = self.props.get(p, {})
            rows.append([d.get(i, math.nan) for i in range(self.n)])
        return rows


def load(name: str) -> Fixture:
    fx = Fixture(name)
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, _, rest = line.partition(" ")
            if head == "n":
                fx.n = int(rest)
            elif head == "concept":
                toks = rest.split()
                fx.concepts[int(toks[0])] = {int(t) for t in toks[1:]}
            elif head == "role":
                toks = rest.split()
                fx.roles[int(toks[0])] = [tuple(int(x) for x in t.split(">")) for t in toks[1:]]
            elif head == "prop":
                toks = rest.split()
                fx.props[int(toks[0])] = {int(t.split("=")[0]): float(t.split("=")[1]) for t in toks[1:]}
            elif head == "pos":
                fx.pos = {int(t) for t in rest.split()}
            elif head == "neg":
                fx.neg = {int(t) for t in rest.split()}
            elif head == "query":
                q, _, ans = rest.partition("=>")
                inst, _, cnt = ans.partition("|")
                fx.queries.append((q.strip(), {int(t) for t in inst.split()},
                                   tuple(int(t) for t in cnt.split())))
            else:
                raise ValueError(line)
    return fx


def fixtures() -> List[str]:
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))
