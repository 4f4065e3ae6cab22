"""Card-name parsing for the test fixtures: rank A,2..10,J,Q,K + suit C,D,H,S -> id 4*rank+suit."""
RANKS = ["A", "2", "3", "4", "5", "6", "7", "8", "9", "10", "J", "Q", "K"]
SUITS = "CDHS"


def card(name: str) -> int:
    return 4 * RANKS.index(name[:-1]) + SUITS.index(name[-1])


def mask(names) -> int:
    m = 0
    for n in names:
        m |= 1 << card(n)
    return m


def name(c: int) -> str:
    return RANKS[c >> 2] + SUITS[c & 3]


def parse_game(path):
    """Worked-game fixture -> (pool ids, hands[6] = (alex ids, bob ids), rows, cleanup, final)."""
    pool, hands, rows, cleanup, final = None, [None] * 6, [], None, None
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        f = line.split()
        if f[0] == "pool":
            pool = [card(x) for x in f[1:]]
        elif f[0] == "hands":
            r = int(f[1])
            bar = f.index("|")
            hands[r] = ([card(x) for x in f[2:bar]], [card(x) for x in f[bar + 1:]])
        elif f[0] == "cleanup":
            cleanup = [int(x) for x in f[1:7]] + [f[7]]
        elif f[0] == "final":
            final = int(f[1])
        else:
            rnd, trn, ply = (int(x) for x in f[0].split("_"))
            pick = 0 if f[2] == "-" else mask(f[2].split(","))
            cols = [int(x) for x in f[3:10]]
            rows.append(dict(round=rnd, turn=trn, ply=ply, lay=card(f[1]), pick=pick, acl=cols[0], bcl=cols[1],
                             apt=cols[2], bpt=cols[3], asr=cols[4], bsr=cols[5], delta=cols[6], L=f[10], CL=f[11]))
    return pool, hands, rows, cleanup, final


def deck_from_game(pool, hands):
    deck = list(pool)
    for a, b in hands:
        deck += a + b
    return deck
